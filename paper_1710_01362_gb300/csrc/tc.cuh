// Blackwell (sm_103a) fifth-generation tensor-core primitives: tcgen05.mma with operands in
// shared memory and the accumulator in tensor memory (TMEM), completion tracked by an
// mbarrier, and the tile GEMM of a complex contraction computed as a real GEMM.
//
// Complex as real.  A complex product Y[r][i] = sum_k Z[r][k] M[i][k] is the real GEMM
//   Yre[r][2i + c] = sum_{k, c'} Zre[r][2k + c'] Bre[2i + c][2k + c']
// with Zre[r][2k] = Re Z, Zre[r][2k + 1] = Im Z and the 2 x 2 block of M[i][k] = a + ib
//   Bre[2i][2k] = a,  Bre[2i][2k + 1] = -b,  Bre[2i + 1][2k] = b,  Bre[2i + 1][2k + 1] = a,
// so that the accumulator row r holds (Re, Im) of Y[r][i] interleaved.
//
// Split precision (FP32 accumulation in TMEM):
//   TF32X3: x = h + l, h = tf32(x), l = tf32(x - h); Y = Zh Bh + Zh Bl + Zl Bh (kind::tf32)
//   BF16X3: x = b0 + b1 + b2, b_j = bf16(x - b_0 - ... - b_{j-1});
//           Y = the six products b_i c_j with i + j <= 2 (kind::f16, bf16 operands)
// Both keep about 22-24 significant bits of every operand (the FP32 level), against 11 (TF32)
// or 8 (BF16) for a single product.
//
// Shared-memory operand layout (no swizzle, K-major): a core matrix is 8 rows x 16 bytes stored
// contiguously (row q of it at 16 q).  Core matrices adjacent along K are LBO = 128 bytes apart,
// core matrices adjacent along the rows (M for A, N for B) are SBO = 128 * (K / E) bytes apart,
// E = 16 / sizeof(element).  One MMA covers 32 bytes of K (two core matrices).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace ttns {
namespace tc {

enum Kind : int { KIND_TF32X3 = 1, KIND_BF16X3 = 2, KIND_BF16X1 = 3 };

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// sm_100-family shared-memory matrix descriptor (no swizzle)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of the sm_100 family; swizzle bits 61-63 = 0
  return d;
}

// instruction descriptor: FP32 accumulator, A and B K-major, dense
// fmt: 2 = TF32 (kind::tf32), 1 = BF16 (kind::f16)
__host__ __device__ constexpr uint32_t idesc(uint32_t fmt, int M, int N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}
// arrives on the mbarrier once every MMA issued so far by this thread has completed
__device__ __forceinline__ void commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes become visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Bounded wait for the phase with the given parity to complete; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, long long spin_limit) {
  const uint32_t a = smem_u32(mbar);
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > spin_limit) return false;
  }
}

// TMEM allocation by one full warp; the base address is written to *dst (shared memory)
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t base, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(ncols) : "memory");
}
// 16 consecutive 32-bit columns of this warp's 32 lanes (lane = accumulator row)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// tcgen05.ld of 8 columns without the wait: the registers are valid only after
// tmem_wait_ld(), and each group of them must then pass through tmem_pin8() so that no use is
// moved above the wait (volatile asm statements keep their order)
__device__ __forceinline__ void tmem_ld8_nowait(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_pin8(uint32_t* r) {
  asm volatile("" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]));
}

// ---------------------------------------------------------------- operand split and layout
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// byte offset of element (row, k) in a K-major no-swizzle operand with K elements per row
// (K a multiple of E = 16 / esize) and element size esize
__device__ __forceinline__ uint32_t kmaj_off(int row, int k, int K, int esize) {
  const int E = 16 / esize;
  return (uint32_t)((row >> 3) * (K / E) * 128 + (k / E) * 128 + (row & 7) * 16 + (k % E) * esize);
}

// Writes the split parts of value x at (row, k) of the operand planes (plane stride pstride bytes)
template <int KIND>
__device__ __forceinline__ void put_split(unsigned char* base, uint32_t pstride, int row, int k, int K, double x) {
  if constexpr (KIND == KIND_TF32X3) {
    const float f = (float)x;
    const float h = to_tf32(f);
    const float l = to_tf32(f - h);
    const uint32_t o = kmaj_off(row, k, K, 4);
    *reinterpret_cast<float*>(base + o) = h;
    *reinterpret_cast<float*>(base + pstride + o) = l;
  } else {
    const __nv_bfloat16 b0 = __double2bfloat16(x);
    const double r1 = x - (double)__bfloat162float(b0);
    const __nv_bfloat16 b1 = __double2bfloat16(r1);
    const double r2 = r1 - (double)__bfloat162float(b1);
    const __nv_bfloat16 b2 = __double2bfloat16(r2);
    const uint32_t o = kmaj_off(row, k, K, 2);
    *reinterpret_cast<__nv_bfloat16*>(base + o) = b0;
    *reinterpret_cast<__nv_bfloat16*>(base + pstride + o) = b1;
    *reinterpret_cast<__nv_bfloat16*>(base + 2 * pstride + o) = b2;
  }
}
template <int KIND>
__device__ __forceinline__ void put_split_f(unsigned char* base, uint32_t pstride, int row, int k, int K, float x) {
  if constexpr (KIND == KIND_BF16X1) {
    *reinterpret_cast<__nv_bfloat16*>(base + kmaj_off(row, k, K, 2)) = __float2bfloat16_rn(x);
  } else if constexpr (KIND == KIND_TF32X3) {
    const float h = to_tf32(x);
    const float l = to_tf32(x - h);
    const uint32_t o = kmaj_off(row, k, K, 4);
    *reinterpret_cast<float*>(base + o) = h;
    *reinterpret_cast<float*>(base + pstride + o) = l;
  } else {
    const __nv_bfloat16 b0 = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(b0);
    const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(b1);
    const __nv_bfloat16 b2 = __float2bfloat16_rn(r2);
    const uint32_t o = kmaj_off(row, k, K, 2);
    *reinterpret_cast<__nv_bfloat16*>(base + o) = b0;
    *reinterpret_cast<__nv_bfloat16*>(base + pstride + o) = b1;
    *reinterpret_cast<__nv_bfloat16*>(base + 2 * pstride + o) = b2;
  }
}

template <int KIND> struct Split;
template <> struct Split<KIND_TF32X3> { static constexpr int parts = 2, esize = 4, kstep = 8; };
template <> struct Split<KIND_BF16X3> { static constexpr int parts = 3, esize = 2, kstep = 16; };
// a single BF16 product (no split): inference-grade, 8 significant bits per operand
template <> struct Split<KIND_BF16X1> { static constexpr int parts = 1, esize = 2, kstep = 16; };

// Issues D (+)= A B^T for one K chunk: A planes (M = 128 rows x K), B planes (N rows x K), K a
// multiple of the MMA's K step.  Split products: TF32X3 {hh, hl, lh}; BF16X3 {00, 01, 10, 02, 11,
// 20}.  Called by one thread; `acc` = 0 starts a fresh accumulation with the chunk's first MMA.
template <int KIND>
__device__ __forceinline__ void issue_chunk(uint32_t d_tmem, const unsigned char* A, uint32_t a_plane,
                                            const unsigned char* B, uint32_t b_plane, int N, int K, bool acc) {
  using S = Split<KIND>;
  const uint32_t E = 16 / S::esize;
  const uint32_t lbo = 128, a_sbo = 128u * (uint32_t)(K / (int)E), b_sbo = a_sbo;
  const uint32_t id = idesc(KIND == KIND_TF32X3 ? 2u : 1u, 128, N);
  const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
  constexpr int NP = KIND == KIND_TF32X3 ? 3 : 6;
  constexpr int pa[6] = {0, 0, 1, 0, 1, 2};
  constexpr int pb[6] = {0, 1, 0, 2, 1, 0};
  bool first = !acc;
  for (int k0 = 0; k0 < K; k0 += S::kstep) {
    const uint32_t koff = (uint32_t)(k0 / (int)E) * 128u;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const uint64_t da = sdesc(a0 + pa[q] * a_plane + koff, lbo, a_sbo);
      const uint64_t db = sdesc(b0 + pb[q] * b_plane + koff, lbo, b_sbo);
      if constexpr (KIND == KIND_TF32X3)
        mma_tf32(d_tmem, da, db, id, first ? 0u : 1u);
      else
        mma_f16(d_tmem, da, db, id, first ? 0u : 1u);
      first = false;
    }
  }
}

// Issues the split products of one MMA K step (k-step index ks of the staged chunk) into a
// fresh accumulator at column d_tmem: the small products first, the hi*hi product last, so that
// the accumulator is rounded once at full scale.  The tensor core rounds its FP32 accumulation
// toward zero (measured on GB300: about -0.4 ulp per MMA instruction); one full-scale rounding
// per K step, with the steps summed on the CUDA cores in round-to-nearest, keeps the sum within
// the FP32 level instead of drifting by 0.4 ulp per instruction.
template <int KIND>
__device__ __forceinline__ void issue_kstep(uint32_t d_tmem, const unsigned char* A, uint32_t a_plane,
                                            const unsigned char* B, uint32_t b_plane, int N, int K, int ks) {
  using S = Split<KIND>;
  const uint32_t E = 16 / S::esize;
  const uint32_t sbo = 128u * (uint32_t)(K / (int)E);
  const uint32_t id = idesc(KIND == KIND_TF32X3 ? 2u : 1u, 128, N);
  const uint32_t koff = (uint32_t)(ks * S::kstep / (int)E) * 128u;
  const uint32_t a0 = smem_u32(A) + koff, b0 = smem_u32(B) + koff;
  // products ordered from the smallest scale to the largest:
  //   TF32X3 (planes h = 0, l = 1): l*h, h*l, h*h
  //   BF16X3 (planes 0, 1, 2):      2*0, 1*1, 0*2, 1*0, 0*1, 0*0
  constexpr int NP = KIND == KIND_TF32X3 ? 3 : (KIND == KIND_BF16X3 ? 6 : 1);
  constexpr int tf_a[3] = {1, 0, 0}, tf_b[3] = {0, 1, 0};
  constexpr int bf_a[6] = {2, 1, 0, 1, 0, 0}, bf_b[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    const int pa = KIND == KIND_TF32X3 ? tf_a[q] : (KIND == KIND_BF16X3 ? bf_a[q] : 0);
    const int pb = KIND == KIND_TF32X3 ? tf_b[q] : (KIND == KIND_BF16X3 ? bf_b[q] : 0);
    const uint64_t da = sdesc(a0 + pa * a_plane, 128, sbo);
    const uint64_t db = sdesc(b0 + pb * b_plane, 128, sbo);
    if constexpr (KIND == KIND_TF32X3)
      mma_tf32(d_tmem, da, db, id, q == 0 ? 0u : 1u);
    else
      mma_f16(d_tmem, da, db, id, q == 0 ? 0u : 1u);
  }
}

}  // namespace tc
}  // namespace ttns
