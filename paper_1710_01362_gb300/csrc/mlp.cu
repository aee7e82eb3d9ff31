// Kernels of the surrogate network (a multilayer perceptron from Hamiltonian parameters to
// population trajectories): the dense layer products on the tensor cores with fused
// epilogues, the bias gradients, the loss gradient and the Adam update.  The paper has no
// network; it names machine learning among the advances its method builds on
// (Introduction).  These kernels are the training and inference engine of this library's
// surrogate, with the plain TTNS sweep as its fallback.
//
// Layer product C = op(A) op(B) on tcgen05, M tiles of 128 rows and N tiles of 128 columns
// per CTA, K in chunks of four MMA K steps.  Every K step accumulates into its own TMEM
// columns and the steps are summed in shared memory in FP32 round-to-nearest (the tensor
// core's own FP32 accumulation rounds toward zero, about -0.4 ulp per instruction):
//   kind 1 (TF32X3): FP32-level products for training;
//   kind 3 (BF16X1): one BF16 product, for inference.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "../../include/ttns.h"
#include "tc.cuh"

namespace ttns {
void set_last_error(const std::string& msg);

namespace {
constexpr int kNT = 256;
constexpr int kTM = 128;         // rows per CTA (MMA M)
constexpr int kTN = 128;         // columns per CTA (MMA N)
constexpr int kTmem = 512;
constexpr int kSlots = kTmem / kTN;  // K steps per chunk, one accumulator each

// status word of the layer products (TTNS_E_TIMEOUT when a completion wait gave up); a
// file-scope device variable, so that no call allocates (the calls can be captured in a graph)
__device__ int g_mlp_status;

struct GemmArgs {
  int M, N, K;
  const float* A;
  int lda, transA;  // A(m, k) = transA ? A[k * lda + m] : A[m * lda + k]
  const float* B;
  int ldb, transB;  // B(k, n) = transB ? B[n * ldb + k] : B[k * ldb + n]
  float* C;
  int ldc;
  int epi;          // 0 C = AB, 1 C = AB + bias, 2 C = tanh(AB + bias), 3 C = AB * (1 - aux^2)
  const float* aux; // bias (epi 1, 2: N values) or the layer output h (epi 3: M x N, ldc)
  long long spin_limit;
};

template <int KIND>
__global__ void __launch_bounds__(kNT, 1) k_mlp_gemm(GemmArgs g) {
  using S = tc::Split<KIND>;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tbase_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kTM, n0 = blockIdx.y * kTN;
  const int nn = min(kTN, g.N - n0);
  const int Npad = ((nn + 15) / 16) * 16;  // MMA N for this tile
  constexpr int KS = S::kstep;
  const int chunk = kSlots * KS;           // real K per chunk
  const int ktot = ((g.K + KS - 1) / KS) * KS;
  const int ldsum = kTN + 1;
  float* sums = reinterpret_cast<float*>(sm);
  const uint32_t sum_bytes = ((uint32_t)kTM * ldsum * 4u + 1023u) & ~1023u;
  const uint32_t a_plane = (uint32_t)kTM * chunk * S::esize;
  const uint32_t b_plane = (uint32_t)kTN * chunk * S::esize;
  unsigned char* Ap = sm + sum_bytes;
  unsigned char* Bp = Ap + S::parts * a_plane;
  if (warp == 0) tc::tmem_alloc(&tbase_s, kTmem);
  if (tid == 0) tc::mbar_init(&mbar, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = tbase_s;
  const int q4 = warp & 3, half = warp >> 2, my_row = q4 * 32 + lane;
  const int c_lo = half * (Npad / 2), c_hi = c_lo + Npad / 2;
  for (int c = c_lo; c < c_hi; ++c) sums[my_row * ldsum + c] = 0.0f;
  uint32_t phase = 0;
  bool ok = true;
  for (int k0 = 0; k0 < ktot && ok; k0 += chunk) {
    const int kn = min(chunk, ktot - k0);   // a multiple of KS
    // A tile: kTM rows x kn; consecutive threads take consecutive rows (transA) or k
    for (int idx = tid; idx < kTM * kn; idx += kNT) {
      int r, k;
      if (g.transA) { r = idx % kTM; k = idx / kTM; } else { k = idx % kn; r = idx / kn; }
      const int m = m0 + r, kk = k0 + k;
      float v = 0.0f;
      if (m < g.M && kk < g.K) v = g.transA ? g.A[(long long)kk * g.lda + m] : g.A[(long long)m * g.lda + kk];
      tc::put_split_f<KIND>(Ap, a_plane, r, k, kn, v);
    }
    // B tile as N x K (K-major): element (n, k) = B(k, n)
    for (int idx = tid; idx < Npad * kn; idx += kNT) {
      int c, k;
      if (g.transB) { k = idx % kn; c = idx / kn; } else { c = idx % Npad; k = idx / Npad; }
      const int n = n0 + c, kk = k0 + k;
      float v = 0.0f;
      if (c < nn && kk < g.K) v = g.transB ? g.B[(long long)n * g.ldb + kk] : g.B[(long long)kk * g.ldb + n];
      tc::put_split_f<KIND>(Bp, b_plane, c, k, kn, v);
    }
    tc::fence_proxy_async();
    __syncthreads();
    const int nsteps = kn / KS;
    if (tid == 0) {
      tc::fence_after();
      for (int ks = 0; ks < nsteps; ++ks)
        tc::issue_kstep<KIND>(tbase + (uint32_t)(ks * Npad), Ap, a_plane, Bp, b_plane, Npad, kn, ks);
      tc::commit(&mbar);
    }
    const bool w = tc::mbar_wait(&mbar, phase, g.spin_limit);
    tc::fence_after();
    ok = __syncthreads_and(w) != 0;
    if (!ok) break;
    phase ^= 1u;
    const uint32_t lane_base = tbase + ((uint32_t)(q4 * 32) << 16);
    for (int c = c_lo; c < c_hi; c += 8) {
      float acc[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] = 0.0f;
      for (int ks = 0; ks < nsteps; ++ks) {
        float v[8];
        tc::tmem_ld8(lane_base + (uint32_t)(ks * Npad + c), v);
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] += v[j];
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) sums[my_row * ldsum + c + j] += acc[j];
    }
    tc::fence_before();
    __syncthreads();
  }
  if (ok) {
    // epilogue: rows of the tile, columns coalesced (one column per thread, rows in turn)
    for (int idx = tid; idx < kTM * nn; idx += kNT) {
      const int r = idx / nn, c = idx % nn;
      const int m = m0 + r, n = n0 + c;
      if (m >= g.M) continue;
      float v = sums[r * ldsum + c];
      if (g.epi == 1 || g.epi == 2) v += g.aux[n];
      if (g.epi == 2) v = tanhf(v);
      if (g.epi == 3) {
        const float h = g.aux[(long long)m * g.ldc + n];
        v *= 1.0f - h * h;
      }
      g.C[(long long)m * g.ldc + n] = v;
    }
  } else {
    if (tid == 0) atomicCAS(&g_mlp_status, 0, (int)TTNS_E_TIMEOUT);
    tc::mbar_wait(&mbar, phase, g.spin_limit);  // the MMAs in flight finish before TMEM is released
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::tmem_dealloc(tbase, kTmem);
}

// out[n] = sum_m X[m * ld + n] (bias gradients), fixed order per column
__global__ void k_colsum(const float* X, int M, int N, int ld, float* out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.0f;
  for (int m = 0; m < M; ++m) s += X[(long long)m * ld + n];
  out[n] = s;
}

// dy = (y - t) * scale
__global__ void k_diff(const float* y, const float* t, float* dy, long long n, float scale) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dy[i] = (y[i] - t[i]) * scale;
}

__global__ void k_adam(float* p, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

template <int KIND>
cudaError_t launch_gemm(const GemmArgs& g, cudaStream_t st) {
  using S = tc::Split<KIND>;
  const size_t sum_bytes = ((size_t)kTM * (kTN + 1) * 4 + 1023) & ~(size_t)1023;
  const size_t smem = sum_bytes + (size_t)S::parts * (kTM + kTN) * (kSlots * S::kstep) * S::esize;
  cudaError_t e = cudaFuncSetAttribute(k_mlp_gemm<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((g.M + kTM - 1) / kTM, (g.N + kTN - 1) / kTN);
  k_mlp_gemm<KIND><<<grid, kNT, smem, st>>>(g);
  return cudaGetLastError();
}
}  // namespace
}  // namespace ttns

using ttns::set_last_error;

extern "C" ttns_status ttns_mlp_gemm(int kind, int M, int N, int K, const float* A, int lda, int transA,
                                     const float* B, int ldb, int transB, float* C, int ldc, int epilogue,
                                     const float* aux, void* cuda_stream) {
  if (!A || !B || !C || ((epilogue >= 1) && !aux)) {
    set_last_error("ttns_mlp_gemm: NULL pointer");
    return TTNS_E_INVALID;
  }
  if ((kind != 1 && kind != 3) || M < 1 || N < 1 || K < 1 || epilogue < 0 || epilogue > 3 || lda < 1 || ldb < 1 ||
      ldc < N || (!transA && lda < K) || (transA && lda < M) || (!transB && ldb < N) || (transB && ldb < K)) {
    set_last_error("ttns_mlp_gemm: bad kind, size, leading dimension or epilogue");
    return TTNS_E_INVALID;
  }
  ttns::GemmArgs g{M, N, K, A, lda, transA, B, ldb, transB, C, ldc, epilogue, aux, 20000000000LL};
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaError_t e = kind == 1 ? ttns::launch_gemm<ttns::tc::KIND_TF32X3>(g, s) : ttns::launch_gemm<ttns::tc::KIND_BF16X1>(g, s);
  if (e != cudaSuccess) {
    set_last_error(std::string("ttns_mlp_gemm: ") + cudaGetErrorString(e));
    return TTNS_E_CUDA;
  }
  return TTNS_OK;
}

extern "C" ttns_status ttns_mlp_colsum(const float* X, int M, int N, int ld, float* out, void* cuda_stream) {
  if (!X || !out || M < 1 || N < 1 || ld < N) {
    set_last_error("ttns_mlp_colsum: bad arguments");
    return TTNS_E_INVALID;
  }
  ttns::k_colsum<<<(N + 255) / 256, 256, 0, (cudaStream_t)cuda_stream>>>(X, M, N, ld, out);
  return cudaGetLastError() == cudaSuccess ? TTNS_OK : TTNS_E_CUDA;
}

extern "C" ttns_status ttns_mlp_diff(const float* y, const float* t, float* dy, long long n, float scale,
                                     void* cuda_stream) {
  if (!y || !t || !dy || n < 1) {
    set_last_error("ttns_mlp_diff: bad arguments");
    return TTNS_E_INVALID;
  }
  ttns::k_diff<<<(int)std::min<long long>(1024, (n + 255) / 256), 256, 0, (cudaStream_t)cuda_stream>>>(y, t, dy, n, scale);
  return cudaGetLastError() == cudaSuccess ? TTNS_OK : TTNS_E_CUDA;
}

extern "C" ttns_status ttns_mlp_adam(float* p, const float* g, float* m, float* v, long long n, float lr, float beta1,
                                     float beta2, float eps, int step, void* cuda_stream) {
  if (!p || !g || !m || !v || n < 1 || step < 1 || !(lr > 0)) {
    set_last_error("ttns_mlp_adam: bad arguments");
    return TTNS_E_INVALID;
  }
  const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
  ttns::k_adam<<<(int)std::min<long long>(1024, (n + 255) / 256), 256, 0, (cudaStream_t)cuda_stream>>>(
      p, g, m, v, n, lr, beta1, beta2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? TTNS_OK : TTNS_E_CUDA;
}

extern "C" ttns_status ttns_mlp_status(int* device_status, int clear) {
  if (!device_status) return TTNS_E_INVALID;
  if (cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpyFromSymbol(device_status, ttns::g_mlp_status, sizeof(int)) != cudaSuccess)
    return TTNS_E_CUDA;
  if (clear) {
    const int zero = 0;
    if (cudaMemcpyToSymbol(ttns::g_mlp_status, &zero, sizeof(int)) != cudaSuccess) return TTNS_E_CUDA;
  }
  return TTNS_OK;
}
