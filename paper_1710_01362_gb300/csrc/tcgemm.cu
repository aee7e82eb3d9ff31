// Self-test of the tensor-core tile GEMM used by the contractions: a complex product
// Y = Z M^T computed with the split-precision tcgen05 path of tc.cuh on one CTA, so that
// its layout, descriptors and split arithmetic can be checked against an FP64 product on the
// host.  The paper has no counterpart: this checks this library's own building block.
#include <cuda_runtime.h>

#include <string>

#include "../../include/ttns.h"
#include "internal.h"
#include "tc.cuh"

namespace ttns {
void set_last_error(const std::string& msg);

namespace {
constexpr int kKC = 32;       // complex K per chunk (64 real)
constexpr int kNT = 256;
constexpr int kTmemCols = 256;

template <int KIND>
__global__ void __launch_bounds__(kNT, 1)
    k_tc_selftest(const double2* Z, const double2* Mt, double2* Y, int Mrows, int Kc, int Nc, int* status,
                  long long spin_limit) {
  using S = tc::Split<KIND>;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tbase_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int Kr = 2 * kKC;                       // real K of one chunk
  const int Npad = ((2 * Nc + 15) / 16) * 16;   // real N, a multiple of 16 (M = 128)
  const uint32_t a_plane = 128u * Kr * S::esize;
  const uint32_t b_plane = (uint32_t)Npad * Kr * S::esize;
  unsigned char* A = sm;
  unsigned char* B = sm + S::parts * a_plane;
  if (warp == 0) tc::tmem_alloc(&tbase_s, kTmemCols);
  if (tid == 0) tc::mbar_init(&mbar, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = tbase_s;
  uint32_t phase = 0;
  bool ok = true;
  for (int row0 = 0; row0 < Mrows && ok; row0 += 128) {
    for (int kc0 = 0; kc0 < Kc && ok; kc0 += kKC) {
      // A chunk: rows row0.., complex k -> real columns 2k (re), 2k + 1 (im)
      for (int idx = tid; idx < 128 * kKC; idx += kNT) {
        const int r = idx / kKC, k = idx % kKC;
        double2 z = make_double2(0.0, 0.0);
        if (row0 + r < Mrows && kc0 + k < Kc) z = Z[(long long)(row0 + r) * Kc + kc0 + k];
        tc::put_split<KIND>(A, a_plane, r, 2 * k, Kr, z.x);
        tc::put_split<KIND>(A, a_plane, r, 2 * k + 1, Kr, z.y);
      }
      // B chunk: 2 x 2 real blocks of M[i][k] = a + ib: [[a, -b], [b, a]]
      for (int idx = tid; idx < (Npad / 2) * kKC; idx += kNT) {
        const int i = idx / kKC, k = idx % kKC;
        double2 m = make_double2(0.0, 0.0);
        if (i < Nc && kc0 + k < Kc) m = Mt[(long long)i * Kc + kc0 + k];
        tc::put_split<KIND>(B, b_plane, 2 * i, 2 * k, Kr, m.x);
        tc::put_split<KIND>(B, b_plane, 2 * i, 2 * k + 1, Kr, -m.y);
        tc::put_split<KIND>(B, b_plane, 2 * i + 1, 2 * k, Kr, m.y);
        tc::put_split<KIND>(B, b_plane, 2 * i + 1, 2 * k + 1, Kr, m.x);
      }
      tc::fence_proxy_async();
      __syncthreads();
      if (tid == 0) {
        tc::fence_after();
        tc::issue_chunk<KIND>(tbase, A, a_plane, B, b_plane, Npad, Kr, kc0 > 0);
        tc::commit(&mbar);
      }
      ok = tc::mbar_wait(&mbar, phase, spin_limit);
      phase ^= 1u;
      tc::fence_after();
      __syncthreads();
    }
    if (!ok) break;
    // epilogue: warps 0-3 read their 32 accumulator rows, 16 columns at a time
    if (warp < 4) {
      const int r = row0 + warp * 32 + lane;
      for (int c0 = 0; c0 < Npad; c0 += 16) {
        float v[16];
        tc::tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        if (r < Mrows)
#pragma unroll
          for (int j = 0; j < 16; j += 2) {
            const int i = (c0 + j) >> 1;
            if (i < Nc) Y[(long long)r * Nc + i] = make_double2((double)v[j], (double)v[j + 1]);
          }
      }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
  }
  if (!ok) {
    if (tid == 0) atomicCAS(status, 0, (int)TTNS_E_TIMEOUT);
    // the MMAs may still be running: wait once more (bounded) before the TMEM is released
    tc::mbar_wait(&mbar, phase ^ 1u, spin_limit);
  }
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, kTmemCols);
}

template <int KIND>
cudaError_t launch_selftest(const double2* Z, const double2* Mt, double2* Y, int M, int K, int N, int* st) {
  using S = tc::Split<KIND>;
  const int Npad = ((2 * N + 15) / 16) * 16;
  const size_t smem = (size_t)S::parts * (128 + Npad) * (2 * kKC) * S::esize;
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
