// Observables beyond the populations: the energy surfaces of Eq. 3-4 and the bond entropies.
//
// Energy surfaces (Results, section on dynamic energy surfaces).  With the orthogonality
// centre at the root, the root tensor A[r][s] (r = the bond indices, s = the electronic state)
// has the Schmidt form A = sum_k sigma_k phi_k(r) u_k(s) for the bipartition electronic |
// environment: u_k are the eigenvectors of rho_S = A^T conj(A) and phi_k = A conj(u_k) / sigma_k.
// In the basis |phi_k>|l> (bath-major) the effective Hamiltonian is
//   H_eff[(i j), (k l)] = <phi_i, j| H |phi_k, l> = sum_r conj(phi_i(r)) (H_root X_kl)[r][j],
// X_kl[r][s] = phi_k(r) delta_sl, H_root the root's local effective Hamiltonian (its
// environment blocks project H onto the bond basis); V_eff = H_eff - T_eff with T the chains'
// kinetic energy, whose environment blocks come from its own environment pass.
//
// Bond entropies (Results, ER section; Methods): S_e = -sum_a lambda_a ln lambda_a over the
// eigenvalues of the density matrix of bond e (the downward pass of bond densities).
//
// Eigenvalues and eigenvectors of the small Hermitian matrices come from a cyclic Jacobi
// method for complex Hermitian matrices (Golub & Van Loan, "Matrix Computations", the
// symmetric Jacobi method, with a diagonal phase rotation that makes each pivot real first):
// one CTA per matrix, FP64.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace ttns {

namespace {
constexpr int kJT = 256;
}

// Batched complex Hermitian Jacobi.  Matrix b (n_b = ns[b] <= 64) starts at base + offs[b],
// row-major with leading dimension ld[b]; eigenvalues (ascending) go to evals + b * 64, and
// when evecs != nullptr the eigenvectors (columns, in the same order) to evecs + b * 64 * 64
// (leading dimension 64).  Dynamic shared memory: n_max^2 complex, twice with vectors.
__global__ void __launch_bounds__(kJT) k_herm_jacobi(const double2* base, const long long* offs, const int* ns,
                                                     const int* lds, double* evals, double2* evecs, int n_max,
                                                     int max_sweeps) {
  extern __shared__ double2 jsm[];
  const int b = blockIdx.x;
  const int n = ns[b];
  const int ld = lds[b];
  const double2* Ain = base + offs[b];
  double2* A = jsm;
  double2* V = jsm + n_max * n_max;
  const bool vecs = evecs != nullptr;
  __shared__ double s_off, s_diag;
  __shared__ double s_c, s_s;
  __shared__ double2 s_e;
  __shared__ int s_skip;
  for (int idx = threadIdx.x; idx < n * n; idx += kJT) {
    const int r = idx / n, c = idx % n;
    A[r * n_max + c] = Ain[(long long)r * ld + c];
    if (vecs) V[r * n_max + c] = make_double2(r == c ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) {
      double off = 0.0, dg = 0.0;
      for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
          const double2 a = A[r * n_max + c];
          if (r == c) dg += a.x * a.x;
          else off += a.x * a.x + a.y * a.y;
        }
      s_off = off;
      s_diag = dg;
    }
    __syncthreads();
    if (!(s_off > 1e-30 * (s_diag + s_off))) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        __syncthreads();  // every thread has read the previous pivot's values
        if (threadIdx.x == 0) {
          const double2 apq = A[p * n_max + q];
          const double r = sqrt(apq.x * apq.x + apq.y * apq.y);
          s_skip = !(r > 1e-300);
          if (!s_skip) {
            // phase: column q times conj(e), row q times e, so that the pivot becomes r
            s_e = make_double2(apq.x / r, apq.y / r);
            const double app = A[p * n_max + p].x, aqq = A[q * n_max + q].x;
            const double tau = (aqq - app) / (2.0 * r);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            s_c = 1.0 / sqrt(1.0 + t * t);
            s_s = t * s_c;
          }
        }
        __syncthreads();
        if (s_skip) continue;
        const double2 e = s_e;
        const double c = s_c, s = s_s;
        // A <- D^H A D with D_qq = conj(e): column q * conj(e), then row q * e
        for (int k = threadIdx.x; k < n; k += kJT) {
          const double2 a = A[k * n_max + q];
          A[k * n_max + q] = make_double2(a.x * e.x + a.y * e.y, a.y * e.x - a.x * e.y);
          if (vecs) {
            const double2 v = V[k * n_max + q];
            V[k * n_max + q] = make_double2(v.x * e.x + v.y * e.y, v.y * e.x - v.x * e.y);
          }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < n; k += kJT) {
          const double2 a = A[q * n_max + k];
          A[q * n_max + k] = make_double2(a.x * e.x - a.y * e.y, a.x * e.y + a.y * e.x);
        }
        __syncthreads();
        // real rotation in the (p, q) plane: columns, then rows (and the vectors' columns)
        for (int k = threadIdx.x; k < n; k += kJT) {
          const double2 akp = A[k * n_max + p], akq = A[k * n_max + q];
          A[k * n_max + p] = make_double2(c * akp.x - s * akq.x, c * akp.y - s * akq.y);
          A[k * n_max + q] = make_double2(s * akp.x + c * akq.x, s * akp.y + c * akq.y);
          if (vecs) {
            const double2 vkp = V[k * n_max + p], vkq = V[k * n_max + q];
            V[k * n_max + p] = make_double2(c * vkp.x - s * vkq.x, c * vkp.y - s * vkq.y);
            V[k * n_max + q] = make_double2(s * vkp.x + c * vkq.x, s * vkp.y + c * vkq.y);
          }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < n; k += kJT) {
          const double2 apk = A[p * n_max + k], aqk = A[q * n_max + k];
          A[p * n_max + k] = make_double2(c * apk.x - s * aqk.x, c * apk.y - s * aqk.y);
          A[q * n_max + k] = make_double2(s * apk.x + c * aqk.x, s * apk.y + c * aqk.y);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          A[p * n_max + q] = make_double2(0.0, 0.0);
          A[q * n_max + p] = make_double2(0.0, 0.0);
        }
        __syncthreads();
      }
  }
  // ascending order (selection by rank: the count of smaller values, ties by index)
  for (int i = threadIdx.x; i < n; i += kJT) {
    const double di = A[i * n_max + i].x;
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double dj = A[j * n_max + j].x;
      rank += (dj < di) || (dj == di && j < i);
    }
    evals[(long long)b * 64 + rank] = di;
    if (vecs)
      for (int k = 0; k < n; ++k) evecs[(long long)b * 64 * 64 + (long long)k * 64 + rank] = V[k * n_max + i];
  }
}

// phi_k(r) = sum_s A[r][s] conj(U[s][k]) / sig[k] for the kept bath states k < nb
__global__ void k_bath_states(const double2* A, long long R, int n_el, const double2* U, const double* sig, int nb,
                              double2* Phi) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < R * nb;
       idx += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(idx / R);
    const long long r = idx - (long long)k * R;
    double re = 0.0, im = 0.0;
    for (int s = 0; s < n_el; ++s) {
      const double2 a = A[r * n_el + s], u = U[s * nb + k];
      re += a.x * u.x + a.y * u.y;
      im += a.y * u.x - a.x * u.y;
    }
    Phi[(long long)k * R + r] = make_double2(re / sig[k], im / sig[k]);
  }
}

// X[r][s] = phi_k(r) delta_{s l}
__global__ void k_build_x(const double2* Phi, int k, int l, long long R, int n_el, double2* X) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < R * n_el;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long r = idx / n_el;
    const int s = (int)(idx - r * n_el);
    X[idx] = s == l ? Phi[(long long)k * R + r] : make_double2(0.0, 0.0);
  }
}

// per-block partials of out[(i j)] = sum_r conj(phi_i(r)) y[r][j], as (re, im) pairs
__global__ void k_project_partial(const double2* y, const double2* Phi, long long R, int n_el, int nb,
                                  double* partials) {
  const int nv = nb * n_el;
  const long long chunk = (R + gridDim.x - 1) / gridDim.x;
  const long long r0 = blockIdx.x * chunk, r1 = min(R, r0 + chunk);
  for (int o = threadIdx.x; o < nv; o += blockDim.x) {
    const int i = o / n_el, j = o % n_el;
    double re = 0.0, im = 0.0;
    for (long long r = r0; r < r1; ++r) {
      const double2 p = Phi[(long long)i * R + r], v = y[r * n_el + j];
      re += p.x * v.x + p.y * v.y;
      im += p.x * v.y - p.y * v.x;
    }
    partials[(long long)blockIdx.x * 2 * nv + 2 * o] = re;
    partials[(long long)blockIdx.x * 2 * nv + 2 * o + 1] = im;
  }
}

// out[k] = sum over blocks of partials (fixed order); column c of a column-major matrix
__global__ void k_reduce_to(const double* partials, int nblocks, int nval, double* out) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nval; k += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partials[(long long)b * nval + k];
    out[k] = s;
  }
}

__global__ void k_sub(const double* a, const double* b, double* c, int n) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) c[k] = a[k] - b[k];
}

cudaError_t launch_herm_jacobi(const double2* base, const long long* offs, const int* ns, const int* lds, int count,
                               int n_max, double* evals, double2* evecs, cudaStream_t st) {
  const size_t smem = (size_t)n_max * n_max * sizeof(double2) * (evecs ? 2 : 1);
  cudaError_t e = cudaFuncSetAttribute(k_herm_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_herm_jacobi<<<count, kJT, smem, st>>>(base, offs, ns, lds, evals, evecs, n_max, 60);
  return cudaGetLastError();
}

cudaError_t launch_bath_states(const double2* A, long long R, int n_el, const double2* U, const double* sig, int nb,
                               double2* Phi, cudaStream_t st) {
  const int blocks = (int)std::min<long long>(1024, (R * nb + 255) / 256);
  k_bath_states<<<blocks, 256, 0, st>>>(A, R, n_el, U, sig, nb, Phi);
  return cudaGetLastError();
}

cudaError_t launch_build_x(const double2* Phi, int k, int l, long long R, int n_el, double2* X, cudaStream_t st) {
  const int blocks = (int)std::min<long long>(1024, (R * n_el + 255) / 256);
  k_build_x<<<blocks, 256, 0, st>>>(Phi, k, l, R, n_el, X);
  return cudaGetLastError();
}

cudaError_t launch_project(const double2* y, const double2* Phi, long long R, int n_el, int nb, double* partials,
                           int nblocks, double* out, cudaStream_t st) {
  k_project_partial<<<nblocks, 128, 0, st>>>(y, Phi, R, n_el, nb, partials);
  const int nval = 2 * nb * n_el;
  k_reduce_to<<<(nval + 255) / 256, 256, 0, st>>>(partials, nblocks, nval, out);
  return cudaGetLastError();
}

cudaError_t launch_sub(const double* a, const double* b, double* c, int n, cudaStream_t st) {
  k_sub<<<(n + 255) / 256, 256, 0, st>>>(a, b, c, n);
  return cudaGetLastError();
}

}  // namespace ttns
