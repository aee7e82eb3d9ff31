// Self-test of the tensor-core tile GEMM used by the contractions: a complex product
// Y = Z M^T computed with the split-precision tcgen05 path of tc.cuh on one CTA, so that
// its layout, descriptors and split arithmetic can be checked against an FP64 product on the
// host.  The paper has no counterpart: this checks this library's own building block.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "../../include/ttns.h"
#include "internal.h"
#include "tc.cuh"

namespace ttns {
void set_last_error(const std::string& msg);

namespace {
constexpr int kNT = 256;
constexpr int kTmemCols = 512;

// Y = Z Mt^T for one CTA, with the sweep's accumulation scheme: chunks of n_acc MMA K steps,
// one fresh TMEM accumulator per K step (small split products first, hi * hi last), and the
// K steps summed on the CUDA cores in FP32 round-to-nearest in a fixed order.
template <int KIND>
__global__ void __launch_bounds__(kNT, 1)
    k_tc_selftest(const double2* Z, const double2* Mt, double2* Y, int Mrows, int Kc, int Nc, int* status,
                  long long spin_limit) {
  using S = tc::Split<KIND>;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tbase_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int Npad = ((2 * Nc + 15) / 16) * 16;   // real N, a multiple of 16 (M = 128)
  constexpr int KSC = S::kstep / 2;              // complex K per MMA K step
  const int n_acc = min(8, kTmemCols / Npad);
  const int chunk_kc = n_acc * KSC;
  const int ktot = ((Kc + KSC - 1) / KSC) * KSC;
  const int ldsum = Npad + 1;
  float* sums = reinterpret_cast<float*>(sm);
  const uint32_t sum_bytes = ((uint32_t)128 * ldsum * 4u + 1023u) & ~1023u;
  const uint32_t a_plane = 128u * 2 * chunk_kc * S::esize;
  const uint32_t b_plane = (uint32_t)Npad * 2 * chunk_kc * S::esize;
  unsigned char* A = sm + sum_bytes;
  unsigned char* B = A + S::parts * a_plane;
  if (warp == 0) tc::tmem_alloc(&tbase_s, kTmemCols);
  if (tid == 0) tc::mbar_init(&mbar, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = tbase_s;
  const int q4 = warp & 3, half = warp >> 2, my_row = q4 * 32 + lane;
  const int c_lo = half * (Npad / 2), c_hi = c_lo + Npad / 2;
  uint32_t phase = 0;
  bool ok = true;
  for (int row0 = 0; row0 < Mrows && ok; row0 += 128) {
    for (int c = c_lo; c < c_hi; ++c) sums[my_row * ldsum + c] = 0.0f;
    for (int kc0 = 0; kc0 < ktot && ok; kc0 += chunk_kc) {
      const int nk = min(chunk_kc, ktot - kc0);
      const int Kr = 2 * nk;
      for (int idx = tid; idx < 128 * nk; idx += kNT) {
        const int r = idx % 128, k = idx / 128;
        double2 z = make_double2(0.0, 0.0);
        if (row0 + r < Mrows && kc0 + k < Kc) z = Z[(long long)(row0 + r) * Kc + kc0 + k];
        tc::put_split<KIND>(A, a_plane, r, 2 * k, Kr, z.x);
        tc::put_split<KIND>(A, a_plane, r, 2 * k + 1, Kr, z.y);
      }
      // 2 x 2 real blocks of M[i][k] = a + ib: [[a, -b], [b, a]]
      for (int idx = tid; idx < (Npad / 2) * nk; idx += kNT) {
        const int k = idx % nk, i = idx / nk;
        double2 m = make_double2(0.0, 0.0);
        if (i < Nc && kc0 + k < Kc) m = Mt[(long long)i * Kc + kc0 + k];
        tc::put_split<KIND>(B, b_plane, 2 * i, 2 * k, Kr, m.x);
        tc::put_split<KIND>(B, b_plane, 2 * i, 2 * k + 1, Kr, -m.y);
        tc::put_split<KIND>(B, b_plane, 2 * i + 1, 2 * k, Kr, m.y);
        tc::put_split<KIND>(B, b_plane, 2 * i + 1, 2 * k + 1, Kr, m.x);
      }
      tc::fence_proxy_async();
      __syncthreads();
      const int nsteps = nk / KSC;
      if (tid == 0) {
        tc::fence_after();
        for (int ks = 0; ks < nsteps; ++ks)
          tc::issue_kstep<KIND>(tbase + (uint32_t)(ks * Npad), A, a_plane, B, b_plane, Npad, Kr, ks);
        tc::commit(&mbar);
      }
      const bool w = tc::mbar_wait(&mbar, phase, spin_limit);
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
    if (!ok) break;
    const int r = row0 + my_row;
    if (r < Mrows)
      for (int c = c_lo; c < c_hi; c += 2) {
        const int i = c >> 1;
        if (i < Nc) Y[(long long)r * Nc + i] = make_double2((double)sums[my_row * ldsum + c], (double)sums[my_row * ldsum + c + 1]);
      }
    __syncthreads();
  }
  if (!ok) {
    if (tid == 0) atomicCAS(status, 0, (int)TTNS_E_TIMEOUT);
    // the MMAs may still be running: wait once more (bounded) before the TMEM is released
    tc::mbar_wait(&mbar, phase, spin_limit);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::tmem_dealloc(tbase, kTmemCols);
}

template <int KIND>
cudaError_t launch_selftest(const double2* Z, const double2* Mt, double2* Y, int M, int K, int N, int* st) {
  using S = tc::Split<KIND>;
  const int Npad = ((2 * N + 15) / 16) * 16;
  const int n_acc = std::min(8, kTmemCols / Npad);
  const int chunk_kc = n_acc * (S::kstep / 2);
  const size_t sum_bytes = ((size_t)128 * (Npad + 1) * 4 + 1023) & ~(size_t)1023;
  const size_t smem = sum_bytes + (size_t)S::parts * (128 + Npad) * (2 * chunk_kc) * S::esize;
  cudaError_t e = cudaFuncSetAttribute(k_tc_selftest<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_tc_selftest<KIND><<<1, kNT, smem>>>(Z, Mt, Y, M, K, N, st, 4000000000LL);
  return cudaGetLastError();
}
}  // namespace
}  // namespace ttns

extern "C" ttns_status ttns_selftest_tc_gemm(int kind, int M, int K, int N, const double* Z, const double* Mt,
                                             double* Y, int* device_status) {
  using namespace ttns;
  if (!Z || !Mt || !Y || !device_status) {
    set_last_error("ttns_selftest_tc_gemm: NULL argument");
    return TTNS_E_INVALID;
  }
  if ((kind != 1 && kind != 2) || M < 1 || M > 4096 || K < 1 || K > 1024 || N < 1 || N > 64) {
    set_last_error("ttns_selftest_tc_gemm: kind must be 1 (TF32X3) or 2 (BF16X3), 1 <= M <= 4096, "
                   "1 <= K <= 1024, 1 <= N <= 64");
    return TTNS_E_INVALID;
  }
  double2 *dZ = nullptr, *dM = nullptr, *dY = nullptr;
  int* dst = nullptr;
  cudaError_t e = cudaMalloc(&dZ, sizeof(double2) * (size_t)M * K);
  if (e == cudaSuccess) e = cudaMalloc(&dM, sizeof(double2) * (size_t)N * K);
  if (e == cudaSuccess) e = cudaMalloc(&dY, sizeof(double2) * (size_t)M * N);
  if (e == cudaSuccess) e = cudaMalloc(&dst, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(dZ, Z, sizeof(double2) * (size_t)M * K, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dM, Mt, sizeof(double2) * (size_t)N * K, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(dY, 0, sizeof(double2) * (size_t)M * N);
  if (e == cudaSuccess) e = cudaMemset(dst, 0, sizeof(int));
  if (e == cudaSuccess)
    e = kind == 1 ? launch_selftest<tc::KIND_TF32X3>(dZ, dM, dY, M, K, N, dst)
                  : launch_selftest<tc::KIND_BF16X3>(dZ, dM, dY, M, K, N, dst);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(Y, dY, sizeof(double2) * (size_t)M * N, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(device_status, dst, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(dZ);
  cudaFree(dM);
  cudaFree(dY);
  cudaFree(dst);
  if (e != cudaSuccess) {
    set_last_error(std::string("ttns_selftest_tc_gemm: ") + cudaGetErrorString(e));
    return TTNS_E_CUDA;
  }
  return TTNS_OK;
}
