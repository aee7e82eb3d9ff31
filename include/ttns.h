/*
 * ttns.h - C ABI of the GB300 tree-tensor-network-state (TTNS) sweep library.
 *
 * The library runs the real-time sweep of arXiv:1710.01362 ("Multi-dimensional
 * Tensor Network Simulation of Open Quantum Dynamics in Singlet Fission") on
 * one GPU.  The paper's problem statement is the star Hamiltonian (Eq. 2):
 *
 *     H = H_S + sum_i [ Wbar_i ||lambda_i|| (a_i0 + a_i0^+)/sqrt(2) + H_c,i ],
 *     H_c,i = sum_n omega_in a_in^+ a_in + sum_n t_in (a_in^+ a_i,n+1 + h.c.),
 *
 * a tree tensor network state with the electronic system at the root and one
 * bosonic chain per environment (Results, "TTNS for vibronic quantum dynamics";
 * Methods, "Tensor Network States"), optionally with a balanced binary tree of
 * entanglement-renormalisation nodes between the root and the chains, evolved
 * with the time-dependent variational principle (one tensor at a time with its
 * local effective Hamiltonian), starting from the zero-temperature vacuum with
 * one electronic state populated.
 *
 * Conventions (all calls):
 *   - energies in eV, times in fs, hbar = 0.6582119569 eV fs;
 *   - complex arrays are interleaved (re, im) doubles, matrices row-major;
 *   - every input array is copied during the call; the caller keeps ownership;
 *   - output arrays are caller-owned host buffers of the stated size;
 *   - no exception crosses the ABI: every call returns a ttns_status, and
 *     ttns_last_error() gives a one-line reason for the last failure;
 *   - work is ordered on the CUDA stream given in ttns_options (NULL = legacy
 *     default stream); calls that return host data synchronise that stream.
 *   - arguments are validated before anything is allocated: bad sizes, NULL
 *     pointers and non-Hermitian H_S / Wbar (tolerance 1e-12) give TTNS_E_INVALID.
 */
#ifndef TTNS_H
#define TTNS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ttns_tree ttns_tree; /* opaque, library-owned */

typedef enum {
  TTNS_OK = 0,
  TTNS_E_INVALID = 1,       /* bad argument */
  TTNS_E_OOM = 2,           /* device allocation failed */
  TTNS_E_CUDA = 3,          /* a CUDA call failed */
  TTNS_E_NOT_CONVERGED = 4, /* a Krylov exponential did not cover its time step within 64
                               Krylov spaces of dimension krylov_mmax (each space takes the
                               largest s / 2^k, k <= 30, that reaches krylov_tol) */
  TTNS_E_TIMEOUT = 5,       /* a device-side wait gave up (bounded spin) */
  TTNS_E_NONFINITE = 6,     /* a norm became NaN or Inf */
  TTNS_E_IO = 7             /* checkpoint file error */
} ttns_status;

/* Precision of the contractions (H_eff / H_bond applications and environment updates).  In
 * every mode the Krylov basis and recurrence, the small exponential and the observables are
 * FP64.  The QR bond steps and the gauge absorbs are FP64 in TTNS_FP64 and double-single
 * (unevaluated sums of two floats, 48-bit significand, error-free transformations; about
 * 2^-44 relative per operation, FP32's exponent range) in the other modes.
 *   TTNS_FP64    every contraction in FP64;
 *   TTNS_TF32X3  split-precision tensor cores: the H_eff applications of tensors of at least 4096
 *                elements whose terms have one dense factor each are complex GEMMs on tcgen05 with
 *                3xTF32 operands (hi*hi + hi*lo + lo*hi) and FP32 accumulation in tensor memory;
 *                every other contraction in FP32 on the SIMT cores;
 *   TTNS_BF16X3  the same with a 3-way BF16 split and the 6 products of order <= 2^-16;
 *   TTNS_FP32    every contraction in FP32 on the SIMT cores.
 * TTNS_MIXED is TTNS_TF32X3. */
typedef enum {
  TTNS_FP64 = 0,
  TTNS_TF32X3 = 1,
  TTNS_MIXED = 1,
  TTNS_BF16X3 = 2,
  TTNS_FP32 = 3
} ttns_precision;

typedef struct {
  int precision;         /* ttns_precision */
  double krylov_tol;     /* Krylov stopping tolerance, 0 -> 1e-12 */
  int krylov_mmax;       /* maximum Krylov dimension, 0 -> 30 (at most 32) */
  void* cuda_stream;     /* cudaStream_t used by every call, NULL = default stream */
  int er_tree;           /* 1: balanced binary ER tree between the root and the chains */
  int D_er;              /* requested bond dimension between ER nodes (er_tree only; clamped like bond_dim) */
  int init_state;        /* electronic state populated at t = 0 (when psi_el is NULL) */
  const double* psi_el;  /* optional initial electronic amplitudes, n_el complex (copied) */
  int record;            /* 1: keep rho_S after every step in a device trajectory buffer */
  int max_record;        /* capacity of that buffer in steps (0 -> 4096) */
  int cluster_ctas;      /* CTAs per cluster team (0 -> 16) */
  int grid_ctas;         /* CTAs of the persistent grid (0 -> as many as can be co-resident) */
  int grid_threshold;    /* single tree: Krylov exponentials, environment updates and absorbs of tensors
                            with at least this many elements are handled by the whole grid, smaller
                            ones by one cluster (0 -> 16384) */
  long long spin_limit;  /* bound of every device-side wait, in SM clock cycles (0 -> 2e10);
                            a wait that runs out sets TTNS_E_TIMEOUT */
  int profile;           /* 1: accumulate per-op device time (see ttns_counters) */
  int launch_flags;      /* bit 0: launch the persistent kernel as a plain cluster launch, without
                            the cooperative attribute (for tools that do not keep the cluster shape
                            of cooperative launches).  Co-residency of the grid then rests on the
                            grid fitting an otherwise idle GPU; a grid barrier that cannot complete
                            ends in TTNS_E_TIMEOUT.  A launch whose cluster shape or shared memory
                            differs from the plan returns before any work; the next synchronising
                            call repeats it (and every step launched since) once as a plain
                            cluster launch, counted in ttns_counters.launch_fallbacks.
                            bit 1: fault injection for tests: step launches get clusters of one
                            CTA, which the kernel refuses, until that repeat has happened. */
  int qr_grid_threshold; /* single tree: the same choice for the QR bond steps (0 -> 65536); QRs keep a
                            column-serial reduction chain, so they favour the smaller team longer */
  double qr_cutoff;      /* relative null threshold of the QR bond step (0 -> 1e-8): a sub-column whose
                            norm is at most qr_cutoff * ||M||_F is completed by the identity reflector
                            and its content is dropped (see the oracle's QR reading) */
} ttns_options;

/* One tree's Hamiltonian (Eq. 2) and truncation.
 *   n_el            number of electronic (diabatic) states, >= 1
 *   H_S             n_el*n_el complex, Hermitian (shifted internally by -tr(H_S)/n_el)
 *   n_env           number of environments (chains), >= 1 (a power of two >= 2 with er_tree)
 *   W_bar           n_env*n_el*n_el complex, each Hermitian: coupling pattern Wbar_i
 *   rc_coupling     n_env: ||lambda_i|| in eV (reaction-coordinate coupling)
 *   chain_len       n_env: L_i >= 1 sites
 *   chain_omega     n_env pointers to L_i onsite energies omega_in (eV)
 *   chain_hop       n_env pointers to L_i - 1 hoppings t_in (eV) (may be NULL when L_i == 1)
 *   local_dim       n_env: Fock truncation d_i >= 2 of every site of chain i
 *   bond_dim        n_env: requested bond dimension D_i >= 1 along chain i (and to its parent)
 *   obb_dim         NULL, or n_env: optimised boson basis dimension of chain i's sites (0: none).
 *                   With obb_dim[i] > 0 every site of chain i is a tensor joined to a leaf that
 *                   holds its Fock leg (dimension local_dim) by a bond of dimension obb_dim[i]
 *                   (Methods: Fock states per mode compressed to a smaller optimised basis)
 * Bond dimensions are clamped to the largest values with D_e <= product of the
 * other leg dimensions at both ends of every bond, so any request at least as large as
 * the Hilbert space (e.g. 1 << 20) asks for the full bond dimension.  A bond that still
 * exceeds 64 after that clamp gives TTNS_E_INVALID. */
typedef struct {
  int n_el;
  const double* H_S;
  int n_env;
  const double* W_bar;
  const double* rc_coupling;
  const int* chain_len;
  const double* const* chain_omega;
  const double* const* chain_hop;
  const int* local_dim;
  const int* bond_dim;
  const int* obb_dim;
} ttns_problem;

/* Builds one tree and its initial state (electronic state init_state, or psi_el,
 * times the vacuum of every chain site), uploads it to device memory and
 * computes the initial environment blocks.  *out receives the new tree. */
ttns_status ttns_build_tree(const ttns_problem* problem, const ttns_options* opt, ttns_tree** out);

/* Builds n_trees independent trees that are advanced together by one
 * persistent launch (one cluster team per tree at a time). */
ttns_status ttns_build_batch(int n_trees, const ttns_problem* problems, const ttns_options* opt,
                             ttns_tree** out);

/* Host-only planning: validates the problems, builds the trees and the compiled
 * step exactly as ttns_build_* would, checks every table offset, and reports
 * sizes without touching the GPU.  bonds[v] is the clamped bond dimension of
 * node v of tree 0 to its parent (0 for the root). */
typedef struct {
  int n_nodes;
  long long pool_complex;          /* complex elements of the state/operator pool */
  int max_node;                    /* largest tensor (complex elements) */
  int max_bond;                    /* largest leg dimension */
  int instructions_per_step;
  long long work_complex_per_worker;
  double apply_flops_per_step;     /* useful flops of one H_eff / H_bond application of every exponential of a step */
  double env_flops_per_step;       /* useful flops of the environment updates of a step */
  int exponentials_per_step;
  int env_updates_per_step;
  int n_bonds_written;
  int bonds[4096];
} ttns_plan_info;
ttns_status ttns_plan(int n_trees, const ttns_problem* problems, const ttns_options* opt, ttns_plan_info* info);

/* Autotuner of the team shape (the number of CTAs per cluster team; in batched mode this
 * sets how many trees advance concurrently).  For each candidate (n_candidates == 0: 16, 8
 * and 4), builds the tree set with *opt and that cluster size, runs one warm-up step of
 * length dt_fs and times one step with CUDA events, then frees it.  Writes the fastest
 * candidate to *best_cluster_ctas (and its seconds per step when best_seconds_per_step is
 * not NULL); pass it as ttns_options.cluster_ctas to the real build.  Candidates must be in
 * 1..16.  TTNS_E_CUDA when no candidate could run.  Uses the GPU; blocks. */
ttns_status ttns_autotune(int n_trees, const ttns_problem* problems, const ttns_options* opt, double dt_fs,
                          int n_candidates, const int* candidates, int* best_cluster_ctas,
                          double* best_seconds_per_step);

/* Advances every tree by n_steps symmetric one-site TDVP steps of length dt_fs
 * (S(dt/2) followed by its adjoint S*(dt/2)).  Asynchronous on the tree's
 * stream; device-side failures are reported by the next synchronising call. */
ttns_status ttns_step(ttns_tree* tree, double dt_fs, int n_steps);

/* Waits for the tree's stream and returns the device status word. */
ttns_status ttns_sync(ttns_tree* tree);

/* rho_out: n_el*n_el complex, the reduced density matrix of the electronic
 * states of tree tree_idx (Results, populations and coherences). */
ttns_status ttns_reduced_density_matrix(ttns_tree* tree, int tree_idx, double* rho_out);

/* occ_out: sum_i L_i doubles, <a^+ a> of every chain site (chains in order,
 * sites from the reaction coordinate outward); the per-chain totals are their sums. */
ttns_status ttns_occupations(ttns_tree* tree, int tree_idx, double* occ_out);

/* norm and energy <H> (eV, with the shifted H_S) of tree tree_idx. */
ttns_status ttns_observables(ttns_tree* tree, int tree_idx, double* norm, double* energy);

/* Energy surfaces (Eq. 3-4, Results, "Dynamic energy surfaces") of tree tree_idx at the
 * current time.  The bath states |phi_k> are the environment Schmidt vectors of the state for
 * the bipartition electronic | environment (from the root tensor, the orthogonality centre),
 * kept where the Schmidt value exceeds sigma_tol; in the basis |phi_k>|l> (bath-major)
 *   H_eff[(i j), (k l)] = <phi_i, j| H |phi_k, l>,   V_eff = H_eff - T_eff,
 * with T the chains' nuclear kinetic energy,
 *   T = -(1/4) sum_m w_m (a^+ - a)_m^2 - (1/2) sum_m t_m (a^+ - a)_m (a^+ - a)_{m+1}
 * (the normal modes' sum w_n p_n^2 / 2 in the chain basis).  Outputs (caller-owned host
 * buffers): tes and pes, n_bath * n_el ascending eigenvalues of H_eff (total energy surfaces)
 * and V_eff (potential energy surfaces); sigma, the n_el Schmidt values (descending);
 * *n_bath.  Needs n_el <= 16 and n_bath * n_el <= 32 (TTNS_E_INVALID otherwise).  Runs the
 * kinetic energy's environment pass and small FP64 kernels; synchronises the stream. */
ttns_status ttns_energy_surfaces(ttns_tree* tree, int tree_idx, double sigma_tol, double* tes, double* pes,
                                 double* sigma, int* n_bath);

/* Entanglement entropies of tree tree_idx at the current time: S_out[0] is the von Neumann
 * entropy -sum lambda ln lambda of the electronic reduced density matrix (system vs.
 * environment), S_out[v] (v = 1 .. n_nodes - 1) that of the bond between node v and its parent
 * (the eigenvalues of the bond's density matrix from the downward pass from the root).
 * Node numbering as in ttns_node_info.  S_out holds n_nodes doubles (caller-owned). */
ttns_status ttns_bond_entropies(ttns_tree* tree, int tree_idx, double* S_out);

/* Adaptive bond dimension (the paper raises bond dimensions until the dynamics converge;
 * Methods, tensor network states).  Single-tree sets only (else TTNS_E_INVALID).
 * new_bond[v] (v = 0 .. n_nodes - 1, host, caller-owned) is the requested dimension of node v's
 * parent bond; the root's entry and requests not above the current dimension leave a bond as
 * it is, and the requests go through the build's Hilbert-space clamp (a bond above 64 after it
 * gives TTNS_E_INVALID and leaves the tree as it was).  Every grown bond gets zero slices in
 * both of its tensors; grown bonds are taken children first, the child's tensor is made an
 * isometry toward its parent again by the sweep's QR (its zero columns get the identity
 * reflector: the completion rule of the step) and R is absorbed into the parent; then every
 * environment block is rebuilt.  The state, the time, the trajectory record and the counters
 * carry over; the device memory of the tree set is reallocated (the handle stays valid).
 * n_grown (optional) receives the number of grown bonds.  Synchronising. */
ttns_status ttns_grow_bonds(ttns_tree* tree, const int* new_bond, int n_nodes, int* n_grown);

/* The adaptive rule: every parent bond below d_max whose smallest Schmidt weight (eigenvalue
 * of the bond's density matrix, from the downward pass) exceeds eps uses all of its dimension
 * and grows by `step`, up to d_max, through ttns_grow_bonds.  eps >= 0, step >= 1 and
 * d_max >= 1, else TTNS_E_INVALID. */
ttns_status ttns_adapt_bonds(ttns_tree* tree, double eps, int step, int d_max, int* n_grown);

/* Copies the recorded rho_S trajectory of tree tree_idx: out holds
 * max_steps*n_el*n_el complex; *n_written receives the number of steps copied. */
ttns_status ttns_trajectory(ttns_tree* tree, int tree_idx, double* out, int max_steps, int* n_written);

/* Device-side populations of every tree (n_trees*n_el doubles, in tree order)
 * written to dev_out on the tree's stream, without synchronising. */
ttns_status ttns_populations_device(ttns_tree* tree, double* dev_out);

/* Cumulative device counters since the build: Krylov iterations, H_eff / H_bond
 * applications, useful contraction flops (8 per complex multiply-add of the
 * sum-of-products terms), exponentials that hit krylov_mmax. */
typedef struct {
  long long krylov_iters;
  long long applies;
  double contraction_flops;
  long long not_converged;
  long long steps;
  /* with ttns_options.profile = 1: device time per op kind (0 forward exponential,
   * 1 QR, 2 environment update, 3 bond exponential, 4 absorb, 5 record) and team
   * (0 whole grid, 1 cluster), in seconds at the SM clock rate, and op counts */
  double op_seconds[6][2];
  long long op_count[6][2];
  /* phases of the cluster-team Krylov exponentials: 0 operator staging, 1 first
   * factors of two-factor terms, 2 apply + alpha reduction (with the tensor-core path:
   * the pass that sums the result slots), 3 recurrence + beta reduction, 4 small
   * exponential / convergence, 5 final combination, 6 norm, 7 tensor-core tasks */
  double expm_phase_seconds[8];
  /* phases of the cluster-team QRs: 0 copy + norm, 1 column loop (its team reductions),
   * 2 Gram of the reflectors, 3 T and Z, 4 Q and R written back, and inside the column
   * loop 5 reflector and coefficients, 6 trailing update, 7 dots for the next column */
  double qr_phase_seconds[8];
  /* the same two breakdowns for the grid-team (whole-GPU) operations */
  double expm_phase_seconds_grid[8];
  double qr_phase_seconds_grid[8];
  /* launches of the persistent kernel that its launch check refused (no planned cluster
   * shape, e.g. under a profiler) and that were repeated as plain cluster launches */
  long long launch_fallbacks;
  /* phases of the environment updates, [0] cluster and [1] grid teams: 0 operator staging
   * and operand conversion, 1 the H-term and channel applications, 2 the projection onto
   * the tensor (per-CTA partials), 3 the team sum of the partials */
  double env_phase_seconds[2][4];
  /* phases of the tensor-core tasks run by the team's first CTA: 0 operand staging, 1 MMA
   * issue and completion, 2 tensor-memory read-back and sums, 3 result write */
  double tc_phase_seconds[4];
} ttns_counters;
ttns_status ttns_get_counters(ttns_tree* tree, ttns_counters* out);

/* Node tensor access (layout: legs [parent] + [children in order] + [physical],
 * row-major).  ttns_node_info gives the number of nodes of tree tree_idx when
 * node < 0, else node's leg count and dims (dims: up to 8 ints). */
ttns_status ttns_node_info(ttns_tree* tree, int tree_idx, int node, int* n_legs, int* dims, int* n_nodes);
ttns_status ttns_get_node(ttns_tree* tree, int tree_idx, int node, double* out, size_t n_complex);

/* Checkpoints.  ttns_save writes every tree's problem (H_S, patterns, chains, dimensions,
 * ER layout, initial amplitudes), the recording settings, and the whole device state
 * (tensors, environment blocks, trajectory, time, step counters).
 * ttns_load builds a new tree set from such a file alone and restores its state: the problem
 * and the recording settings come from the file; the run options (precision, Krylov
 * settings, stream, team shape) from *opt (NULL = defaults).  *out receives the new tree.
 * ttns_load_state restores a file's state into an existing tree set of the same shape.
 * Tensor contents are not validated on load: a non-finite entry is reported by the next
 * step as TTNS_E_NONFINITE.  A missing, truncated or mismatching file gives TTNS_E_IO. */
ttns_status ttns_save(ttns_tree* tree, const char* path);
ttns_status ttns_load(const char* path, const ttns_options* opt, ttns_tree** out);
ttns_status ttns_load_state(ttns_tree* tree, const char* path);

/* Self-test of the device-side bounded wait (no counterpart in the paper: failure
 * handling of this library).  With spin_limit > 0, a two-CTA barrier is launched in
 * which one CTA never arrives; the other gives up after spin_limit SM cycles and
 * *device_status receives TTNS_E_TIMEOUT.  With spin_limit == 0 both arrive and
 * *device_status receives TTNS_OK.  Uses the legacy default stream. */
ttns_status ttns_selftest_wait_timeout(long long spin_limit, int* device_status);

/* Self-test of the tensor-core tile GEMM behind the split-precision contractions (no
 * counterpart in the paper: a check of this library's building block).  Computes the complex
 * product Y[m][n] = sum_k Z[m][k] Mt[n][k] on one CTA with tcgen05 MMAs, as a real GEMM of 2 x 2
 * blocks with FP32 accumulation in tensor memory, in split precision kind = 1 (TF32X3: 3 TF32
 * products) or kind = 2 (BF16X3: 6 BF16 products of a 3-way split).  Z: M x K, Mt: N x K,
 * Y: M x N complex (interleaved doubles, row-major, host buffers); 1 <= M <= 4096,
 * 1 <= K <= 1024, 1 <= N <= 64.  *device_status receives TTNS_E_TIMEOUT if a completion
 * wait gave up, else TTNS_OK.  Allocates device memory; synchronises the device. */
ttns_status ttns_selftest_tc_gemm(int kind, int M, int K, int N, const double* Z, const double* Mt, double* Y,
                                  int* device_status);

/* Surrogate-network kernels (no counterpart in the paper, which names machine learning
 * among the advances its method builds on (Introduction) but gives no network: these train
 * and run this library's multilayer perceptron from Hamiltonian parameters to population
 * trajectories, with the TTNS sweep as its fallback).  All pointers are caller-owned device
 * memory (FP32, row-major); every call is enqueued on cuda_stream (NULL = legacy default
 * stream), allocates nothing and does not synchronise.
 *
 * ttns_mlp_gemm: C = op(A) op(B) on the tensor cores (tcgen05), M x N, inner dimension K,
 *   op(A)(m, k) = transA ? A[k * lda + m] : A[m * lda + k],
 *   op(B)(k, n) = transB ? B[n * ldb + k] : B[k * ldb + n],
 *   kind 1: 3xTF32 products (FP32-level, for training); kind 3: one BF16 product (inference).
 *   Every MMA K step has its own tensor-memory accumulator and the steps are summed in FP32
 *   round-to-nearest.  epilogue: 0 C = AB; 1 C = AB + aux[n] (bias); 2 C = tanh(AB + aux[n]);
 *   3 C = AB * (1 - aux[m * ldc + n]^2) (backward through tanh, aux = that layer's output).
 * ttns_mlp_colsum: out[n] = sum_m X[m * ld + n] (bias gradients), fixed order.
 * ttns_mlp_diff:   dy[i] = (y[i] - t[i]) * scale (gradient of the squared loss).
 * ttns_mlp_adam:   one Adam step (Kingma & Ba) on n parameters p with gradients g and moments
 *   m, v at step number step >= 1.
 * ttns_mlp_status: synchronises the device and reads the status word of the layer products
 *   (TTNS_E_TIMEOUT if a completion wait gave up), clearing it when clear != 0.
 * Bad sizes or NULL pointers give TTNS_E_INVALID before anything is launched. */
ttns_status ttns_mlp_gemm(int kind, int M, int N, int K, const float* A, int lda, int transA, const float* B, int ldb,
                          int transB, float* C, int ldc, int epilogue, const float* aux, void* cuda_stream);
ttns_status ttns_mlp_colsum(const float* X, int M, int N, int ld, float* out, void* cuda_stream);
ttns_status ttns_mlp_diff(const float* y, const float* t, float* dy, long long n, float scale, void* cuda_stream);
ttns_status ttns_mlp_adam(float* p, const float* g, float* m, float* v, long long n, float lr, float beta1, float beta2,
                          float eps, int step, void* cuda_stream);
ttns_status ttns_mlp_status(int* device_status, int clear);

/* Electronic reduced density matrix from a root tensor in caller-owned device
 * memory, allocating nothing (the paper has no counterpart: this is for callers
 * that cannot call cudaMalloc, e.g. code running inside another framework's
 * locked memory pool or on threads that must not trigger an allocation).
 *   d_root   device pointer: rows x n_el complex (interleaved doubles), row-major,
 *            the electronic leg last (the root layout of ttns_get_node)
 *   rows     product of the root's bond dimensions, >= 1, with rows * n_el < 2^24
 *   n_el     1..16 electronic states
 *   d_rho    device pointer: n_el x n_el complex output, rho[s][s'] = sum_r A[r][s] conj(A[r][s'])
 *   cuda_stream  stream the two kernels are enqueued on (NULL = legacy default stream)
 * Partial sums go to a fixed 1 MiB scratch array owned by the library on every
 * device that loads it; n_el > 16 is rejected with TTNS_E_INVALID.  The first call
 * on a device looks up that array's address (with the device current): make it
 * before any stream capture, and do not use the call across a cudaDeviceReset (the
 * remembered address belongs to the context that was reset).  Calls share the array, so calls that overlap on the
 * GPU race; each call overwrites all the partials it uses.  Asynchronous. */
ttns_status ttns_rho_from_root_noalloc(const double* d_root, long long rows, int n_el, double* d_rho,
                                       void* cuda_stream);

/* Message of the last failing call made by the calling host thread (thread-local storage
 * owned by the library; valid until that thread's next failing call). */
const char* ttns_last_error(void);
/* Waits for the tree set's stream, then releases every device buffer and the handle.
 * NULL is accepted (no-op).  The handle must not be used afterwards. */
void ttns_free(ttns_tree* tree);

/* Environments from per-mode couplings (host, FP64; Results, "Interface to TTNS": modes with
 * similar coupling patterns are grouped by weighted k-means with k-means++ seeding, each
 * group becomes one chain of Eq. 2).  W: n_modes * n_el * n_el complex, mode n's coupling
 * matrix W_n (Eq. 1).  Every mode's pattern Wbar_n = W_n / ||W_n||_F is a point of 2 n_el^2
 * reals with weight ||W_n||_F^2; W and -W are one direction, so a mode meets a centre c
 * aligned by the sign of <x, c>, at the distance ||x||^2 + ||c||^2 - 2 |<x, c>|.  Lloyd
 * iterations start from the centres init[0..k) (mode indices, the caller's k-means++ draw),
 * assign each mode to the nearest centre (ties to the lower index), move each centre to the
 * weighted mean of its sign-aligned modes (an empty cluster keeps its centre), and stop when
 * no assignment changes or after max_iter.
 * Outputs (caller-owned): assign (n_modes cluster indices), W_bar (k * n_el * n_el complex,
 * the centres at Frobenius norm 1), lambda (n_modes: Re <Wbar_assign(n), W_n>_F, the mode's
 * strength along its environment's pattern), *iterations.  Feed each environment's modes
 * (frequencies, lambda) to ttns_chain_from_modes for its chain. */
ttns_status ttns_cluster_modes(int n_modes, int n_el, const double* W, int k, const int* init, int max_iter,
                               int* assign, double* W_bar, double* lambda, int* iterations);

/* Chain maps (host, FP64).  ttns_chain_ohmic: closed form for the Ohmic density
 * J(w) = 2 pi alpha w exp(-w/omega_c) (Laguerre weight): ||lambda|| = 2 omega_c
 * sqrt(alpha), omega_n = omega_c (2n+2), t_n = omega_c sqrt((n+1)(n+2)).
 * ttns_chain_from_modes: Lanczos tridiagonalisation of diag(omega) from
 * lambda/||lambda|| with full re-orthogonalisation (L <= n_modes).
 * Outputs: rc (1 double), onsite (L), hop (L-1), caller-owned. */
ttns_status ttns_chain_ohmic(double alpha, double omega_c, int L, double* rc, double* onsite, double* hop);
ttns_status ttns_chain_from_modes(int n_modes, const double* omega, const double* lambda, int L, double* rc,
                                  double* onsite, double* hop);

#ifdef __cplusplus
}
#endif
#endif /* TTNS_H */
