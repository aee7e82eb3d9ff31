// Device side of the TTNS sweep: one persistent cooperative kernel that runs the
// compiled one-site TDVP step (Results, "TTNS for vibronic quantum dynamics":
// every tensor evolved in turn with its local effective Hamiltonian) for n steps.
//
// Execution model (GB300: 152 SMs, FP64 at about 1/80 of the FP32 rate with a long
// dependent latency, and the FP64 <-> FP32 conversions on the same narrow pipe; hardware
// cluster barriers ~0.2 us; the software grid barrier meets at the cluster barrier first):
//   * a "team" executes one instruction: either one thread-block cluster (hardware
//     barrier; small tensors, and every QR below the QR threshold) or the whole grid
//     (software barrier; Krylov exponentials, environment updates and absorbs of tensors
//     above the grid threshold);
//   * in batched mode every cluster advances its own trees independently;
//   * reductions are deterministic: per-CTA partials, then a fixed-order sum
//     that every CTA computes identically (no floating-point atomics);
//   * every spin-wait is bounded and reports TTNS_E_TIMEOUT instead of hanging.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <type_traits>

#include "internal.h"
#include "tc.cuh"

namespace cg = cooperative_groups;

namespace ttns {

#define NT 256
#define NWARP (NT / 32)
#define HBAR_EVFS 0.6582119569

// status codes mirrored from ttns.h
#define ST_TIMEOUT 5
#define ST_NOT_CONVERGED 4
#define ST_NONFINITE 6
#define ST_LAUNCH 3       // the launch did not have the cluster shape / shared memory it was planned for

__constant__ double c_inv[256];       // 1/n, c_inv[0] = 0
__constant__ double c_invfact[128];   // 1/n!

// ------------------------------------------------------------------ complex helpers
template <typename T> struct C2;
template <> struct C2<double> { using t = double2; };
template <> struct C2<float> { using t = float2; };

template <typename T>
__device__ __forceinline__ typename C2<T>::t ld(const double2* p) {
  double2 v = *p;
  typename C2<T>::t r;
  r.x = (T)v.x;
  r.y = (T)v.y;
  return r;
}
template <typename T>
__device__ __forceinline__ typename C2<T>::t cvt(double2 v) {
  typename C2<T>::t r;
  r.x = (T)v.x;
  r.y = (T)v.y;
  return r;
}
template <typename T>
__device__ __forceinline__ typename C2<T>::t cvt(float2 v) {
  typename C2<T>::t r;
  r.x = (T)v.x;
  r.y = (T)v.y;
  return r;
}

template <typename T>
__device__ __forceinline__ void cmac(typename C2<T>::t& acc, typename C2<T>::t a, typename C2<T>::t b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

// ------------------------------------------------------------------ teams
struct Team {
  int kind;      // TEAM_GRID / TEAM_CLUSTER
  int rank;      // CTA rank in the team
  int size;      // CTAs in the team
  double* red;   // two partial buffers, red_stride doubles each
  long long red_stride;
  int parity;
  Ctl* ctl;
  long long spin_limit;
  int csize;     // CTAs per thread-block cluster (the grid team reduces per cluster first)
  __device__ int nthr() const { return size * NT; }
  __device__ int gtid() const { return rank * NT + (int)threadIdx.x; }
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_volatile_int(const int* p) { return *(volatile const int*)p; }

__device__ void set_status(Ctl* ctl, int st, int where, int node) {
  if (atomicCAS(&ctl->status, 0, st) == 0) {
    ctl->err_where = where;
    ctl->err_node = node;
  }
}

// software barrier over all CTAs of the grid; bounded.  Hierarchical: the CTAs of each
// thread-block cluster meet at the hardware cluster barrier, one thread per cluster arrives
// at the global counter and waits for the generation to change, and a second cluster barrier
// releases its cluster.  The cluster barriers' release/acquire and the global release/acquire
// pair order every CTA's writes before the barrier with every CTA's reads after it.  A launch
// without clusters is a grid of one-CTA clusters.
__device__ void grid_sync(Ctl* ctl, long long spin_limit) {
  cg::cluster_group cl = cg::this_cluster();
  const unsigned csz = cl.num_blocks();
  if (csz > 1) cl.sync(); else __syncthreads();
  if (cl.block_rank() == 0 && threadIdx.x == 0) {
    const unsigned nclu = gridDim.x / csz;
    unsigned g = ld_acquire(&ctl->bar_gen);
    __threadfence();
    unsigned prev = atomicAdd(&ctl->bar_count, 1u);
    if (prev == nclu - 1) {
      atomicExch(&ctl->bar_count, 0u);
      __threadfence();
      asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(&ctl->bar_gen), "r"(g + 1) : "memory");
    } else {
      // bounded wait; the bound applies to time without progress of the working cluster
      long long t0 = clock64();
      unsigned seen = *(volatile unsigned*)&ctl->progress;
      while (ld_acquire(&ctl->bar_gen) == g) {
        if (ld_volatile_int(&ctl->status) != 0) break;
        const unsigned pr = *(volatile unsigned*)&ctl->progress;
        if (pr != seen) {
          seen = pr;
          t0 = clock64();
        }
        if (clock64() - t0 > spin_limit) {
          set_status(ctl, ST_TIMEOUT, 100, -1);
          break;
        }
      }
    }
    __threadfence();
  }
  if (csz > 1) cl.sync(); else __syncthreads();
}

__device__ __forceinline__ void team_sync(Team& tm) {
  if (tm.kind == TEAM_CLUSTER) {
    cg::this_cluster().sync();
  } else {
    grid_sync(tm.ctl, tm.spin_limit);
  }
}

// warp sum with a fixed order; every lane returns lane 0's value
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return __shfl_sync(0xffffffffu, v, 0);
}

template <int NV>
__device__ __forceinline__ void warp_sum_n(double* v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
}

// Sum of V values (a power of two <= 16) over a warp with V - 1 + 5 - log2(V) additions per
// lane instead of 5 V: the first log2(V) butterfly levels exchange half of the remaining
// values, the rest are plain.  Lane L returns the total of value warp_reduce_vid<V>(L); the
// FP64 pipe, which also runs these additions, is the narrow one on this part.
template <int V>
__device__ __forceinline__ int warp_reduce_vid(int lane) {
  int vid = 0;
#pragma unroll
  for (int n = V, off = 16; n > 1; n >>= 1, off >>= 1)
    if (lane & off) vid += n / 2;
  return vid;
}
template <int V>
__device__ __forceinline__ double warp_reduce_t(double* v) {
  const int lane = threadIdx.x & 31;
  int off = 16;
#pragma unroll
  for (int n = V; n > 1; n >>= 1, off >>= 1) {
    const bool hi = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < n / 2; ++i) {
      const double send = hi ? v[i] : v[i + n / 2];
      const double keep = hi ? v[i + n / 2] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  double t = v[0];
#pragma unroll
  for (; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
  return t;
}

// All-reduce of nv per-thread values over the team (up to four per barrier).  Deterministic
// and identical on every CTA.  Inside a CTA the 256 values go through shared memory to warp
// 0, which adds them in a fixed tree (7 additions per lane, then one transposing butterfly
// for all values, instead of a butterfly per value on every warp: the additions run on the
// narrow FP64 pipe).  Cluster teams push each CTA's totals into every peer's shared memory
// before the cluster barrier, so that after it the sums come from local shared memory; the
// grid team goes through global memory.
static_assert(NT == 256, "team_allreduce assumes 256 threads per CTA");
__device__ void team_allreduce4(Team& tm, double* v, int nv) {
  __shared__ double s_all[4][NT];
  __shared__ double s_out[4];
  __shared__ double s_recv[2][16][4];  // [parity][source rank][value] (cluster teams, <= 16 CTAs)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < 4; ++i) s_all[i][threadIdx.x] = i < nv ? v[i] : 0.0;
  __syncthreads();
  double tot[4] = {0.0, 0.0, 0.0, 0.0};  // this CTA's totals (warp 0, every lane)
  if (warp == 0) {
    double t[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const double* a = s_all[i];
      t[i] = ((a[lane] + a[lane + 32]) + (a[lane + 64] + a[lane + 96])) +
             ((a[lane + 128] + a[lane + 160]) + (a[lane + 192] + a[lane + 224]));
    }
    const double r = warp_reduce_t<4>(t);  // lanes 0, 8, 16, 24: values 0..3
#pragma unroll
    for (int i = 0; i < 4; ++i) tot[i] = __shfl_sync(0xffffffffu, r, 8 * i);
  }
  if (tm.kind == TEAM_CLUSTER) {
    cg::cluster_group cl = cg::this_cluster();
    if (warp == 0 && lane < tm.size) {
      double* dst = cl.map_shared_rank(&s_recv[tm.parity][tm.rank][0], lane);
#pragma unroll
      for (int i = 0; i < 4; ++i) dst[i] = tot[i];
    }
    cl.sync();
    if (warp == 0) {
      double t[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) t[i] = lane < tm.size ? s_recv[tm.parity][lane][i] : 0.0;
      const double r = warp_reduce_t<4>(t);
      if ((lane & 7) == 0) s_out[lane >> 3] = r;
    }
  } else {
    double* buf = tm.red + (long long)tm.parity * tm.red_stride;
    if (threadIdx.x == 0)
#pragma unroll
      for (int i = 0; i < 4; ++i) buf[tm.rank * 4 + i] = tot[i];
    team_sync(tm);
    if (warp == 0) {
      double t[4] = {0.0, 0.0, 0.0, 0.0};
      for (int r = lane; r < tm.size; r += 32)
#pragma unroll
        for (int i = 0; i < 4; ++i) t[i] += buf[r * 4 + i];
      const double r = warp_reduce_t<4>(t);
      if ((lane & 7) == 0) s_out[lane >> 3] = r;
    }
  }
  __syncthreads();
  for (int i = 0; i < nv; ++i) v[i] = s_out[i];
  tm.parity ^= 1;
}

__device__ void team_allreduce(Team& tm, double* v, int nv) {
  for (int i0 = 0; i0 < nv; i0 += 4) team_allreduce4(tm, v + i0, nv - i0 < 4 ? nv - i0 : 4);
}

// Multi-value all-reduce: every CTA has written nval partial doubles at
// part[rank * nval ...] (in the current parity buffer); after the call out[k]
// holds the fixed-order sum over CTAs, written by exactly one thread of the team.
// The caller must team_sync before reading `out` from other CTAs.
__device__ double* team_partials(Team& tm) { return tm.red + (long long)tm.parity * tm.red_stride; }

__device__ void team_finish_multi(Team& tm, int nval, double* out, double scale) {
  team_sync(tm);
  double* buf = team_partials(tm);
  for (int k = tm.gtid(); k < nval; k += tm.nthr()) {
    double s = 0;
    for (int r = 0; r < tm.size; ++r) s += buf[(long long)r * nval + k];
    out[k] = s * scale;
  }
  tm.parity ^= 1;
  team_sync(tm);
}

// ------------------------------------------------------------------ sum-of-products apply
// Position decomposition of flat index idx along leg l.
// n / d for 0 <= n < 2^24 through a float reciprocal, corrected to the exact quotient
// (the float estimate is within 2 of it); 64-bit integer division is emulated and slow.
__device__ __forceinline__ int fdivu(int n, int d, float inv) {
  int q = __float2int_rz((float)n * inv);
  int r = n - q * d;
  if (r < 0) { --q; r += d; }
  if (r < 0) { --q; r += d; }
  if (r >= d) { ++q; r -= d; }
  if (r >= d) { ++q; }
  return q;
}

struct LegPos {
  long long base;  // idx - i * stride
  int i;
};
__device__ __forceinline__ LegPos leg_pos(const NodeDesc& nd, int l, long long idx) {
  const int st = nd.strides[l], D = nd.dims[l];
  const int n = (int)idx;
  const int q = fdivu(n, st, nd.inv_strides[l]);
  const int i = q - fdivu(q, D, nd.inv_dims[l]) * D;
  return LegPos{(long long)(n - i * st), i};
}

// y_i = sum_k M[i][k] x[base + k*stride] with four independent accumulators.  M is a row
// of a dims x dims matrix, either staged in shared memory (compute type) or in the pool.
template <typename T, typename MT, typename XT>
__device__ __forceinline__ typename C2<T>::t mode_dot(const MT* row, int D, const XT* x, long long base, int stride) {
  using V = typename C2<T>::t;
  V a0, a1, a2, a3;
  a0.x = a0.y = a1.x = a1.y = a2.x = a2.y = a3.x = a3.y = (T)0;
  const XT* xp = x + base;
  int k = 0;
  for (; k + 3 < D; k += 4) {
    const V m0 = cvt<T>(row[k]), m1 = cvt<T>(row[k + 1]), m2 = cvt<T>(row[k + 2]), m3 = cvt<T>(row[k + 3]);
    const V x0 = cvt<T>(xp[(long long)k * stride]), x1 = cvt<T>(xp[(long long)(k + 1) * stride]);
    const V x2 = cvt<T>(xp[(long long)(k + 2) * stride]), x3 = cvt<T>(xp[(long long)(k + 3) * stride]);
    cmac<T>(a0, m0, x0);
    cmac<T>(a1, m1, x1);
    cmac<T>(a2, m2, x2);
    cmac<T>(a3, m3, x3);
  }
  for (; k < D; ++k) cmac<T>(a0, cvt<T>(row[k]), cvt<T>(xp[(long long)k * stride]));
  a0.x += a1.x + (a2.x + a3.x);
  a0.y += a1.y + (a2.y + a3.y);
  return a0;
}

// Staging of one op's operands in shared memory.  Every node's operators (the
// environment blocks flowing into it and its constant operators) are contiguous in the
// pool, so an op stages one or two regions with asynchronous copies (cp.async), plus its
// term list; a factor's shared-memory slot is its offset inside the staged regions.  The
// matrices are staged in the compute type: FP64 from the pool, or FP32 from its mirror.
extern __shared__ __align__(16) unsigned char dyn_smem[];

// operator data in the compute type: the FP64 pool, or its FP32 mirror
template <typename T>
__device__ __forceinline__ const typename C2<T>::t* ops(const KernelParams& P);
template <>
__device__ __forceinline__ const double2* ops<double>(const KernelParams& P) { return P.pool; }
template <>
__device__ __forceinline__ const float2* ops<float>(const KernelParams& P) { return P.pool32; }

struct OpStage {
  Term terms[TTNS_MAX_TERMS];
  Factor chans[16];
  long long a_off, b_off;  // pool offsets of the staged regions
  int a_n, b_n;            // staged elements of each (a prefix when the region is larger)
  int end;                 // first free double2 of the dynamic shared memory
};

// one staging record per CTA, shared by every op (ops run one at a time)
__shared__ OpStage s_os;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <typename T>
__device__ void stage_op(const KernelParams& P, const Instr& I, const TermList& L, const Factor* chans, int nchan,
                         OpStage& os) {
  // half of the dynamic shared memory for matrices (in the compute type), half for vectors
  using V = typename C2<T>::t;
  const long long cap = P.smem_bytes / (long long)sizeof(V) / 2;
  __syncthreads();
  if (threadIdx.x == 0) {
    const long long an = I.rega_len < cap ? I.rega_len : cap;
    const long long rest = cap - an;
    const long long bn = I.regb_len < rest ? I.regb_len : rest;
    os.a_off = I.rega_off;
    os.b_off = I.regb_off;
    os.a_n = (int)an;
    os.b_n = (int)bn;
    // end of the staged matrices in 16-byte units, rounded up to 32 bytes
    const long long bytes = (an + bn) * (long long)sizeof(V);
    os.end = (int)((((bytes + 15) / 16) + 1) & ~1LL);
  }
  const int nt = L.count < TTNS_MAX_TERMS ? L.count : TTNS_MAX_TERMS;
  for (int t = threadIdx.x; t < nt; t += NT) os.terms[t] = P.terms[L.first + t];
  for (int b = threadIdx.x; b < nchan && b < 16; b += NT) os.chans[b] = chans[b];
  __syncthreads();
  if constexpr (std::is_same<T, double>::value) {
    double2* sm = reinterpret_cast<double2*>(dyn_smem);
    for (int k = threadIdx.x; k < os.a_n; k += NT) cp_async16(sm + k, P.pool + os.a_off + k);
    for (int k = threadIdx.x; k < os.b_n; k += NT) cp_async16(sm + os.a_n + k, P.pool + os.b_off + k);
    cp_async_wait_all();
  } else {
    // from the FP32 mirror (a double -> float conversion per element would run on the FP64
    // pipe) with asynchronous 8-byte copies: every copy of a thread is in flight at once
    float2* sm = reinterpret_cast<float2*>(dyn_smem);
    for (int k = threadIdx.x; k < os.a_n; k += NT) cp_async8(sm + k, P.pool32 + os.a_off + k);
    for (int k = threadIdx.x; k < os.b_n; k += NT) cp_async8(sm + os.a_n + k, P.pool32 + os.b_off + k);
    cp_async_wait_all();
  }
  __syncthreads();
}

// shared-memory position of n pool elements starting at pool offset off, or -1
__device__ __forceinline__ int staged_at(const OpStage& os, long long off, long long n) {
  long long e = off - os.a_off;
  if (e >= 0 && e + n <= os.a_n) return (int)e;
  e = off - os.b_off;
  if (e >= 0 && e + n <= os.b_n) return os.a_n + (int)e;
  return -1;
}

__device__ __forceinline__ int fslot(const OpStage& os, const Factor& f, int D) {
  const long long need = (long long)D * D;
  long long e = f.mat - os.a_off;
  if (e >= 0 && e + need <= os.a_n) return (int)e;
  e = f.mat - os.b_off;
  if (e >= 0 && e + need <= os.b_n) return os.a_n + (int)e;
  return -1;
}

// Input vector staged in shared memory (compute type) after the matrices, when it fits.
template <typename T>
__device__ typename C2<T>::t* vec_smem(const KernelParams& P, const OpStage& os, long long N) {
  using V = typename C2<T>::t;
  const long long avail = P.smem_bytes - (long long)os.end * (long long)sizeof(double2);
  if (N * (long long)sizeof(V) > avail) return nullptr;
  return reinterpret_cast<V*>(dyn_smem + (long long)os.end * sizeof(double2));
}

template <typename T>
__device__ void stage_vector(typename C2<T>::t* dst, const double2* src, long long N) {
  __syncthreads();
  long long k = threadIdx.x;
  for (; k + 3 * NT < N; k += 4 * NT) {  // four independent loads in flight per thread
    const double2 a = src[k], b = src[k + NT], c = src[k + 2 * NT], d = src[k + 3 * NT];
    dst[k] = cvt<T>(a);
    dst[k + NT] = cvt<T>(b);
    dst[k + 2 * NT] = cvt<T>(c);
    dst[k + 3 * NT] = cvt<T>(d);
  }
  for (; k < N; k += NT) dst[k] = cvt<T>(src[k]);
  __syncthreads();
}

// A compute-type vector copied into shared memory with asynchronous copies.
__device__ void stage_copy(float2* dst, const float2* src, long long N) {
  __syncthreads();
  for (long long k = threadIdx.x; k < N; k += NT) cp_async8(dst + k, src + k);
  cp_async_wait_all();
  __syncthreads();
}

// One factor applied at output idx: sum_k M[i][k] x[idx + (k - i) * stride] along the factor's leg.
template <typename T, typename XT>
__device__ __forceinline__ typename C2<T>::t factor_dot(const KernelParams& P, const NodeDesc& nd, const Factor& f,
                                                        const OpStage& os, const XT* x, long long idx) {
  const LegPos lp = leg_pos(nd, f.leg, idx);
  const int D = nd.dims[f.leg];
  if (f.nnz > 0) {
    using V = typename C2<T>::t;
    V acc;
    acc.x = acc.y = (T)0;
    const int sl = staged_at(os, f.sp, 2LL * D * f.nnz);
    if (sl >= 0) {  // the table staged with the node's operators, in the compute type
      const V* tab = reinterpret_cast<const V*>(dyn_smem) + sl;
      const V* vals = tab + lp.i * f.nnz;
      const V* cols = tab + D * f.nnz + lp.i * f.nnz;
      for (int e = 0; e < f.nnz; ++e) {
        const int k = (int)cols[e].x;
        cmac<T>(acc, vals[e], cvt<T>(x[lp.base + (long long)k * nd.strides[f.leg]]));
      }
      return acc;
    }
    const V* vals = ops<T>(P) + f.sp + (long long)lp.i * f.nnz;
    const V* cols = ops<T>(P) + f.sp + (long long)D * f.nnz + (long long)lp.i * f.nnz;
    for (int e = 0; e < f.nnz; ++e) {
      const int k = (int)cols[e].x;
      cmac<T>(acc, vals[e], cvt<T>(x[lp.base + (long long)k * nd.strides[f.leg]]));
    }
    return acc;
  }
  const int slot = fslot(os, f, D);
  if (slot >= 0) {  // staged in the compute type
    const typename C2<T>::t* sm = reinterpret_cast<const typename C2<T>::t*>(dyn_smem) + slot;
    return mode_dot<T>(sm + lp.i * D, D, x, lp.base, nd.strides[f.leg]);
  }
  return mode_dot<T>(ops<T>(P) + f.mat + (long long)lp.i * D, D, x, lp.base, nd.strides[f.leg]);
}

// Direct two-factor term at idx: the sparse factor's few entries, each times the dense
// factor applied at the shifted position.
template <typename T, typename XT>
__device__ __forceinline__ typename C2<T>::t direct_dot(const KernelParams& P, const NodeDesc& nd, const Term& T_,
                                                        const OpStage& os, const XT* x, long long idx) {
  using V = typename C2<T>::t;
  const Factor& sf = T_.f[T_.sparse_f];
  const Factor& df = T_.f[1 - T_.sparse_f];
  const LegPos lp = leg_pos(nd, sf.leg, idx);
  const int Ds = nd.dims[sf.leg];
  V acc;
  acc.x = acc.y = (T)0;
  const int sl = staged_at(os, sf.sp, 2LL * Ds * sf.nnz);
  if (sl >= 0) {  // staged table (compute type)
    const V* tab = reinterpret_cast<const V*>(dyn_smem) + sl;
    const V* vals = tab + lp.i * sf.nnz;
    const V* cols = tab + Ds * sf.nnz + lp.i * sf.nnz;
    for (int e = 0; e < sf.nnz; ++e) {
      const V v = vals[e];
      if (v.x == (T)0 && v.y == (T)0) continue;
      const long long idx2 = lp.base + (long long)((int)cols[e].x) * nd.strides[sf.leg];
      const V d = factor_dot<T>(P, nd, df, os, x, idx2);
      cmac<T>(acc, v, d);
    }
    return acc;
  }
  const V* vals = ops<T>(P) + sf.sp + (long long)lp.i * sf.nnz;
  const V* cols = ops<T>(P) + sf.sp + (long long)Ds * sf.nnz + (long long)lp.i * sf.nnz;
  for (int e = 0; e < sf.nnz; ++e) {
    const V v = vals[e];
    if (v.x == (T)0 && v.y == (T)0) continue;
    const long long idx2 = lp.base + (long long)((int)cols[e].x) * nd.strides[sf.leg];
    const V d = factor_dot<T>(P, nd, df, os, x, idx2);
    cmac<T>(acc, v, d);
  }
  return acc;
}

// Stage 1: tmp[t] = first factor of two-stage term t applied to x (tmp in the compute type)
template <typename T, typename XT>
__device__ void apply_stage1(const KernelParams& P, Team& tm, const NodeDesc& nd, const XT* x, const TermList& L,
                             typename C2<T>::t* tmp, long long tstride, const OpStage& os) {
  const int t0 = L.count - L.n2;
  const long long N = nd.size;
  for (long long idx = tm.gtid(); idx < N; idx += tm.nthr()) {
    for (int t = 0; t < L.n2; ++t) tmp[t * tstride + idx] = factor_dot<T>(P, nd, os.terms[t0 + t].f[0], os, x, idx);
  }
}

// Stage 2 value at idx: one-factor and direct terms on x, second factors on tmp
template <typename T, typename XT>
__device__ __forceinline__ typename C2<T>::t apply_stage2_at(const KernelParams& P, const NodeDesc& nd, const XT* x,
                                                            const TermList& L, const typename C2<T>::t* tmp,
                                                            long long tstride, long long idx, const OpStage& os) {
  typename C2<T>::t acc;
  acc.x = 0;
  acc.y = 0;
  const int n1 = L.count - L.n2 - L.nd;
  for (int t = 0; t < n1; ++t) {
    const auto a = factor_dot<T>(P, nd, os.terms[t].f[0], os, x, idx);
    acc.x += a.x;
    acc.y += a.y;
  }
  for (int t = n1; t < n1 + L.nd; ++t) {
    const auto a = direct_dot<T>(P, nd, os.terms[t], os, x, idx);
    acc.x += a.x;
    acc.y += a.y;
  }
  const int t0 = L.count - L.n2;
  for (int t = 0; t < L.n2; ++t) {
    const auto a = factor_dot<T>(P, nd, os.terms[t0 + t].f[1], os, tmp + t * tstride, idx);
    acc.x += a.x;
    acc.y += a.y;
  }
  return acc;
}

// ------------------------------------------------------------------ tridiagonal exponential
// u = exp(-i s T) e_0 for the real symmetric tridiagonal T (diag a[0..m), off-diagonal
// b[1..m) with b[k] coupling k-1 and k), by a Chebyshev expansion on the Gershgorin
// interval: exp(-i z X) = J_0(z) + 2 sum_n (-i)^n J_n(z) T_n(X), X = (T - c)/R, z = s R.
// Runs on one warp (lane k holds component k, m <= 32); FP64 throughout.
__device__ __noinline__ void texp_warp(const double* a, const double* b, int m, double s, double* ure, double* uim) {
  const int lane = threadIdx.x & 31;
  const bool on = lane < m;
  double ak = on ? a[lane] : 0.0;
  double bk = (on && lane > 0) ? b[lane] : 0.0;
  double bk1 = (lane + 1 < m) ? b[lane + 1] : 0.0;
  double lo = on ? ak - fabs(bk) - fabs(bk1) : 1e300;
  double hi = on ? ak + fabs(bk) + fabs(bk1) : -1e300;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  lo = __shfl_sync(0xffffffffu, lo, 0);
  hi = __shfl_sync(0xffffffffu, hi, 0);
  const double c = 0.5 * (hi + lo);
  double R = 0.5 * (hi - lo);
  double vre = (lane == 0) ? 1.0 : 0.0, vim = 0.0;  // current vector (complex)
  if (R > 0.0) {
    // sub-steps so that |z| <= 8 per Chebyshev expansion
    double zt = fabs(s) * R;
    if (!(zt < 1e4)) zt = 0.0;  // non-finite input: the caller reports it
    int nsub = (int)ceil(zt / 8.0);
    if (nsub < 1) nsub = 1;
    const double z = s * R / nsub;     // signed
    const double az = fabs(z);
    // truncation: the last coefficient ~ 2 (|z|/2)^K / K! below 1e-17
    int K = 1;
    {
      double term = 1.0;
      while (K < 64 && (term > 1e-18 || K < (int)az + 2)) {
        term *= 0.5 * az * c_inv[K];
        ++K;
      }
    }
    // Bessel J_n(|z|) for n = lane and lane + 32 via the power series in Horner form
    double J[2];
    const double y = -0.25 * az * az;
    int jmax = (int)(3.0 * az + 8.0);
    if (jmax > 24) jmax = 24;
    for (int h = 0; h < 2; ++h) {
      const int n = lane + 32 * h;
      double acc = 1.0;
      if (n < K) {
        for (int j = jmax; j >= 1; --j) acc = fma(acc * y, c_inv[j] * c_inv[j + n], 1.0);
        J[h] = acc * pow(0.5 * az, (double)n) * c_invfact[n];
      } else {
        J[h] = 0.0;
      }
    }
    const double dk = on ? (ak - c) / R : 0.0;
    const double ek = on ? bk / R : 0.0;
    const double fk = on ? bk1 / R : 0.0;
    for (int sub = 0; sub < nsub; ++sub) {
      // Chebyshev on the complex vector v: w = sum_n coef_n T_n(X) v with real T_n
      double t0r = vre, t0i = vim;
      double accr = 0.0, acci = 0.0;
      double tmr = 0.0, tmi = 0.0;   // T_{n-1} v
      double tr = t0r, ti = t0i;     // T_n v
      for (int n = 0; n < K; ++n) {
        const double Jn = __shfl_sync(0xffffffffu, J[n >> 5], n & 31);
        double cr, ci;  // coef_n = (n ? 2 : 1) (-i sgn(z))^n J_n(|z|)
        const double w = (n ? 2.0 : 1.0) * Jn;
        const int q = n & 3;
        const bool neg = z < 0.0;
        // (-i)^n for z > 0; (+i)^n for z < 0
        if (q == 0) { cr = w; ci = 0.0; }
        else if (q == 2) { cr = -w; ci = 0.0; }
        else if ((q == 1) != neg) { cr = 0.0; ci = -w; }
        else { cr = 0.0; ci = w; }
        accr = fma(cr, tr, fma(-ci, ti, accr));
        acci = fma(cr, ti, fma(ci, tr, acci));
        // next Chebyshev vector
        double trl = __shfl_up_sync(0xffffffffu, tr, 1), til = __shfl_up_sync(0xffffffffu, ti, 1);
        double trr = __shfl_down_sync(0xffffffffu, tr, 1), tir = __shfl_down_sync(0xffffffffu, ti, 1);
        if (lane == 0) { trl = 0.0; til = 0.0; }
        if (lane + 1 >= m) { trr = 0.0; tir = 0.0; }
        double xr = fma(dk, tr, fma(ek, trl, fk * trr));
        double xi = fma(dk, ti, fma(ek, til, fk * tir));
        double nr, ni;
        if (n == 0) { nr = xr; ni = xi; }
        else { nr = fma(2.0, xr, -tmr); ni = fma(2.0, xi, -tmi); }
        if (!on) { nr = 0.0; ni = 0.0; }
        tmr = tr; tmi = ti;
        tr = nr; ti = ni;
      }
      vre = accr;
      vim = acci;
    }
  }
  // global phase exp(-i s c)
  double sn, cs;
  sincos(-s * c, &sn, &cs);
  const double rr = vre * cs - vim * sn;
  const double ri = vre * sn + vim * cs;
  if (on) { ure[lane] = rr; uim[lane] = ri; }
}

// Sum of nval doubles over the team, in a fixed order, identical on every CTA.  `mine`
// holds this CTA's partials in shared memory and `out` receives the sums (shared memory).
// Cluster teams read the other CTAs' partials through distributed shared memory: callers
// alternate between two `mine` buffers, so that one cluster barrier per call suffices (a
// buffer is rewritten only after the next call's barrier, which every reader has passed).
// Grid teams go through the global partial buffers.
__device__ void team_reduce_vec(Team& tm, const double* mine, double* out, int nval) {
  __syncthreads();
  if (tm.kind == TEAM_CLUSTER) {
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();
    for (int k = threadIdx.x; k < nval; k += NT) {
      // the 16 peers' values loaded together, then added in a fixed tree (depth 4)
      double a[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) a[r] = r < tm.size ? *cl.map_shared_rank(mine + k, r) : 0.0;
#pragma unroll
      for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
        for (int r = 0; r < w; ++r) a[r] += a[r + w];
      out[k] = a[0];
    }
  } else {
    // grid team: each cluster first sums its CTAs' partials through distributed shared memory
    // (the values split over the cluster's CTAs, each value added in a fixed tree), the cluster
    // totals go to global memory, and after the grid barrier every CTA adds the few cluster
    // totals in a fixed order.  Every CTA computes the same sums.
    cg::cluster_group cl = cg::this_cluster();
    const int cs = tm.csize;
    const int crank = (int)cl.block_rank();
    const int cid = tm.rank / cs;
    const int ncl = tm.size / cs;
    double* buf = team_partials(tm);
    cl.sync();
    for (int k = crank * NT + threadIdx.x; k < nval; k += cs * NT) {
      double a[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) a[r] = r < cs ? *cl.map_shared_rank(mine + k, r) : 0.0;
#pragma unroll
      for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
        for (int r = 0; r < w; ++r) a[r] += a[r + w];
      buf[(long long)cid * nval + k] = a[0];
    }
    team_sync(tm);
    for (int k = threadIdx.x; k < nval; k += NT) {
      double s = 0.0;
      for (int c = 0; c < ncl; ++c) s += buf[(long long)c * nval + k];
      out[k] = s;
    }
    tm.parity ^= 1;
  }
  __syncthreads();
}

// Butterfly sum of NV values over a warp (every lane ends with a full sum; lane 0's is used).
// ------------------------------------------------------------------ Lanczos exponential
struct KrylovShared {
  double alpha[TTNS_KMAX + 1];
  double beta[TTNS_KMAX + 2];   // beta[j] couples j-1 and j
  double scale[TTNS_KMAX + 1];  // q_j = scale[j] * K_j
  double ure[TTNS_KMAX];
  double uim[TTNS_KMAX];
  double rv[2][2 * (TTNS_KMAX + 1)];  // reorthogonalisation: per-CTA dot partials (alternating)
  double rvo[2 * (TTNS_KMAX + 1)];    // and their team sums
  int flag;
};
__shared__ KrylovShared s_ks;

// Full reorthogonalisation of the FP64 path (the oracle's Lanczos does the same): two
// classical Gram-Schmidt passes of w = K_{j+1} against q_i = scale_i K_i, i = 0..j,
//   w <- w - sum_i <q_i, w> q_i,  <q_i, w> = scale_i <K_i, w>.
// The dots are team sums (fixed order); each pass costs one team reduction.  The
// functions return this thread's share of |w|^2 after the second pass.
//
// Vectors in global memory, elements idx = gtid + k * nthr (op_expm):
__device__ double reorth_strided(Team& tm, long long N, const double2* x, const double2* Kb, long long kv,
                                 double2* W, int j, KrylovShared& ks) {
  __shared__ double s_wp[NWARP][16];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  auto Kp = [&](int i) -> const double2* { return i == 0 ? x : Kb + (long long)(i - 1) * kv; };
  double nrm = 0.0;
  for (int pass = 0; pass < 2; ++pass) {
    double* mine = ks.rv[pass];
    for (int i0 = 0; i0 <= j; i0 += 8) {
      const int ni = min(8, j + 1 - i0);
      double acc[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) acc[q] = 0.0;
      for (long long idx = tm.gtid(); idx < N; idx += tm.nthr()) {
        const double2 w = W[idx];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          if (q < ni) {
            const double2 k = Kp(i0 + q)[idx];
            acc[2 * q] = fma(k.x, w.x, fma(k.y, w.y, acc[2 * q]));
            acc[2 * q + 1] = fma(k.x, w.y, fma(-k.y, w.x, acc[2 * q + 1]));
          }
        }
      }
      warp_sum_n<16>(acc);
      if (lane == 0)
#pragma unroll
        for (int q = 0; q < 16; ++q) s_wp[warp][q] = acc[q];
      __syncthreads();
      if (threadIdx.x < 2 * ni) {
        double sum = 0.0;
        for (int w = 0; w < NWARP; ++w) sum += s_wp[w][threadIdx.x];
        mine[2 * i0 + threadIdx.x] = sum;
      }
      __syncthreads();
    }
    team_reduce_vec(tm, mine, ks.rvo, 2 * (j + 1));
    nrm = 0.0;
    for (long long idx = tm.gtid(); idx < N; idx += tm.nthr()) {
      double2 w = W[idx];
      for (int i = 0; i <= j; ++i) {
        const double sc = ks.scale[i];
        const double cr = sc * ks.rvo[2 * i], ci = sc * ks.rvo[2 * i + 1];  // <q_i, w>
        const double2 k0 = Kp(i)[idx];
        const double2 k = make_double2(sc * k0.x, sc * k0.y);             // q_i
        w.x -= cr * k.x - ci * k.y;
        w.y -= cr * k.y + ci * k.x;
      }
      W[idx] = w;
      nrm = fma(w.x, w.x, fma(w.y, w.y, nrm));
    }
  }
  return nrm;
}

// Slices in shared memory, elements [0, n_own) of every K_i slice (op_expm_cluster):
__device__ double reorth_slices(Team& tm, const double2* basis, long long S, int n_own, int j, KrylovShared& ks) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double2* Kj1 = basis + (long long)(j + 1) * S;
  double2* W = const_cast<double2*>(Kj1);
  double nrm = 0.0;
  for (int pass = 0; pass < 2; ++pass) {
    double* mine = ks.rv[pass];
    __syncthreads();  // w was written with the thread-strided mapping; the dots read it per lane
    for (int i = warp; i <= j; i += NWARP) {  // warp per basis vector, lanes over the slice
      const double2* Ki = basis + (long long)i * S;
      double acc[2] = {0.0, 0.0};
      for (int e = lane; e < n_own; e += 32) {
        const double2 k = Ki[e], w = W[e];
        acc[0] = fma(k.x, w.x, fma(k.y, w.y, acc[0]));
        acc[1] = fma(k.x, w.y, fma(-k.y, w.x, acc[1]));
      }
      warp_sum_n<2>(acc);
      if (lane == 0) {
        mine[2 * i] = acc[0];
        mine[2 * i + 1] = acc[1];
      }
    }
    team_reduce_vec(tm, mine, ks.rvo, 2 * (j + 1));
    nrm = 0.0;
    for (int e = threadIdx.x; e < n_own; e += NT) {
      double2 w = W[e];
      for (int i = 0; i <= j; ++i) {
        const double sc = ks.scale[i];
        const double cr = sc * ks.rvo[2 * i], ci = sc * ks.rvo[2 * i + 1];  // <q_i, w>
        const double2 k0 = basis[(long long)i * S + e];
        const double2 k = make_double2(sc * k0.x, sc * k0.y);             // q_i
        w.x -= cr * k.x - ci * k.y;
        w.y -= cr * k.y + ci * k.x;
      }
      W[e] = w;
      nrm = fma(w.x, w.x, fma(w.y, w.y, nrm));
    }
  }
  return nrm;
}


struct PhaseClock {
  long long t;
  bool on;
  bool grid;  // phases of grid-team ops go to their own counters
  __device__ void start(bool enable, bool grid_team = false) {
    on = enable;
    grid = grid_team;
    t = clock64();
  }
  __device__ void lap(Ctl* ctl, int phase) {
    if (!on) return;
    const long long now = clock64();
    atomicAdd(grid ? &ctl->phase_cycles_grid[phase] : &ctl->phase_cycles[phase], (unsigned long long)(now - t));
    t = now;
  }
};

// Cluster-resident Krylov exponential for small nodes.  Each CTA of the cluster owns a
// contiguous slice of every Krylov vector in its shared memory; the full input vector of
// each application is all-gathered through distributed shared memory, every operator is
// staged once, and the only global traffic is the node tensor in and out.  The arithmetic
// is the same as op_expm's (same recurrence, same reductions, same convergence and
// substep rules).
template <typename T>
__device__ __noinline__ bool op_expm_cluster(const KernelParams& P, Team& tm, const Instr& I, double tau) {
  using V = typename C2<T>::t;
  KrylovShared& ks = s_ks;
  OpStage& os = s_os;
  PhaseClock pc;
  pc.start(P.profile && tm.rank == 0 && threadIdx.x == 0);
  const NodeDesc nd = P.nodes[I.node];
  const TermList L = P.lists[I.terms];
  const long long N = nd.size;
  const int cs = tm.size;
  const long long S = (N + cs - 1) / cs;           // slice length
  const long long e0 = (long long)tm.rank * S;
  const long long e1 = min(N, e0 + S);
  const int mmax = min(P.mmax, (int)(N < (long long)TTNS_KMAX ? N : (long long)TTNS_KMAX));
  // shared-memory layout after the matrices: [xs: N V][tmp: n2*N V][basis: (mmax+1)*S double2]
  {
    const long long mats = (long long)(I.rega_len + I.regb_len) * sizeof(V);
    long long off = (long long)(N + (long long)L.n2 * N) * sizeof(V);
    off = (off + 15) & ~15LL;
    const long long need = mats + 32 + off + (long long)(mmax + 1) * S * sizeof(double2) + S * (long long)sizeof(V);
    if (need > P.smem_bytes) return false;  // same decision on every CTA (same sizes)
  }
  stage_op<T>(P, I, L, nullptr, 0, os);
  unsigned char* base = dyn_smem + ((long long)os.end * sizeof(double2));
  V* xs = reinterpret_cast<V*>(base);
  V* tmp = xs + N;
  long long off = (long long)(N + (long long)L.n2 * N) * sizeof(V);
  off = (off + 15) & ~15LL;
  double2* basis = reinterpret_cast<double2*>(base + off);
  // mixed precision: the own slice of the current Krylov vector in the compute type, which
  // the other CTAs gather (converted once, by its owner)
  constexpr bool kShadow = !std::is_same<T, double>::value;
  V* kf = reinterpret_cast<V*>(basis + (long long)(mmax + 1) * S);
  cg::cluster_group cl = cg::this_cluster();
  auto Ks = [&](int j) -> double2* { return basis + (long long)j * S; };
  double2* x = P.pool + nd.off;
  double s_rem = I.sign * tau / HBAR_EVFS;
  int total_m = 0, m = 0;
  for (long long e = e0 + threadIdx.x; e < e1; e += NT) Ks(0)[e - e0] = x[e];
  __syncthreads();
  pc.lap(P.ctl, 0);
  for (int chunk = 0; chunk < 64; ++chunk) {
    double v[1] = {0.0};
    for (long long e = e0 + threadIdx.x; e < e1; e += NT) {
      const double2 a = Ks(0)[e - e0];
      v[0] = fma(a.x, a.x, fma(a.y, a.y, v[0]));
      if constexpr (kShadow) kf[e - e0] = cvt<T>(a);
    }
    team_allreduce(tm, v, 1);
    const double beta0 = sqrt(v[0]);
    pc.lap(P.ctl, 6);
    if (!(beta0 > 0.0)) {
      if (!(beta0 == 0.0)) set_status(P.ctl, ST_NONFINITE, I.op, I.node);
      break;
    }
    if (threadIdx.x == 0) {
      ks.scale[0] = 1.0 / beta0;
      ks.beta[0] = 0.0;
    }
    __syncthreads();
    m = 0;
    bool conv = false;
    double bnext = 0.0, lead = 1.0;
    int next_check = 1;
    for (int j = 0; j < mmax; ++j) {
      // all-gather K_j (complete on every CTA: written before the last cluster barrier),
      // from the compute-type slices in mixed precision
      {
        V* src = kShadow ? kf : reinterpret_cast<V*>(Ks(j));
        const float invS = 1.0f / (float)S;
        int e = threadIdx.x;
        for (; e + 3 * NT < (int)N; e += 4 * NT) {
          V a[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int ee = e + q * NT;
            const int r = fdivu(ee, (int)S, invS);
            a[q] = cl.map_shared_rank(src, r)[ee - r * (int)S];
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) xs[e + q * NT] = a[q];
        }
        for (; e < (int)N; e += NT) {
          const int r = fdivu(e, (int)S, invS);
          xs[e] = cl.map_shared_rank(src, r)[e - r * (int)S];
        }
      }
      __syncthreads();
      if (L.n2 > 0) {
        // first factors of the two-stage terms, on the elements that the own slice's second
        // factors read: the slice widened to whole blocks of the second factor's leg (every
        // CTA computes its range from the gathered input; for a factor on the last leg the
        // range is the slice's rows)
        const int t0 = L.count - L.n2;
        for (int t = 0; t < L.n2; ++t) {
          const int l2 = os.terms[t0 + t].f[1].leg;
          const long long blk = (long long)nd.dims[l2] * nd.strides[l2];
          const long long lo = e1 > e0 ? (e0 / blk) * blk : 0;
          const long long hi = e1 > e0 ? min(N, ((e1 - 1) / blk + 1) * blk) : 0;
          for (long long e = lo + threadIdx.x; e < hi; e += NT)
            tmp[t * N + e] = factor_dot<T>(P, nd, os.terms[t0 + t].f[0], os, xs, e);
        }
        __syncthreads();
      }
      pc.lap(P.ctl, 1);
      const double sj = ks.scale[j], bj = ks.beta[j];
      const double sjm = j > 0 ? ks.scale[j - 1] : 0.0;
      double2* W = Ks(j + 1);
      // part[0] = Re <K_j, w>; in mixed precision also part[1] = |w|^2, so that one team
      // reduction gives both alpha_j and beta_{j+1}
      const bool mixed = P.precision != 0;
      double part[3] = {0.0, 0.0, 0.0};
      for (long long e = e0 + threadIdx.x; e < e1; e += NT) {
        const auto a = apply_stage2_at<T>(P, nd, xs, L, tmp, N, e, os);
        const double2 kj = Ks(j)[e - e0];
        double wr = sj * (double)a.x, wi = sj * (double)a.y;
        if (j > 0) {
          const double2 km = Ks(j - 1)[e - e0];
          wr = fma(-bj * sjm, km.x, wr);
          wi = fma(-bj * sjm, km.y, wi);
        }
        W[e - e0] = make_double2(wr, wi);
        part[0] = fma(kj.x, wr, fma(kj.y, wi, part[0]));
        if (mixed) {
          part[1] = fma(wr, wr, fma(wi, wi, part[1]));
          part[2] = fma(kj.x, kj.x, fma(kj.y, kj.y, part[2]));
        }
      }
      team_allreduce(tm, part, mixed ? 3 : 1);
      pc.lap(P.ctl, 2);
      const double aj = part[0] * sj;
      // |w - alpha_j q_j|^2 = |w|^2 - 2 alpha_j^2 + alpha_j^2 |q_j|^2 with |q_j|^2 from the same
      // reduction (the error of an assumed |q_j| = 1 would grow by alpha^2 / beta^2 per step);
      // used unless it cancels (the same decision on every CTA)
      const double nq = sj * sj * part[2];
      const double b2 = part[1] - aj * aj * (2.0 - nq);
      const bool fused = mixed && b2 > 1e-4 * part[1];
      double nrm[1] = {0.0};
      for (long long e = e0 + threadIdx.x; e < e1; e += NT) {
        const double2 kj = Ks(j)[e - e0];
        double2 w = W[e - e0];
        w.x = fma(-aj * sj, kj.x, w.x);
        w.y = fma(-aj * sj, kj.y, w.y);
        W[e - e0] = w;
        if constexpr (kShadow) kf[e - e0] = cvt<T>(w);  // gathered after the next barrier
        nrm[0] = fma(w.x, w.x, fma(w.y, w.y, nrm[0]));
      }
      if (P.precision == 0) nrm[0] = reorth_slices(tm, basis, S, (int)max(0LL, e1 - e0), j, ks);
      if (fused) {
        bnext = sqrt(b2);
        cl.sync();  // the slices of K_{j+1} are complete before any CTA gathers them
      } else {
        team_allreduce(tm, nrm, 1);
        bnext = sqrt(nrm[0]);
      }
      pc.lap(P.ctl, 3);
      if (threadIdx.x == 0) {
        ks.alpha[j] = aj;
        ks.beta[j + 1] = bnext;
        ks.scale[j + 1] = bnext > 0.0 ? 1.0 / bnext : 0.0;
      }
      __syncthreads();
      m = j + 1;
      const double est = bnext * lead;
      lead *= fabs(s_rem) * bnext / (double)m;
      if ((est <= 1e2 * P.tol && m >= next_check) || m == mmax || !(bnext > 0.0)) {
        next_check = m + 1;
        if (threadIdx.x < 32) texp_warp(ks.alpha, ks.beta, m, s_rem, ks.ure, ks.uim);
        __syncthreads();
        const double um = sqrt(ks.ure[m - 1] * ks.ure[m - 1] + ks.uim[m - 1] * ks.uim[m - 1]);
        const double err = bnext * um;
        if (!(err == err)) {
          set_status(P.ctl, ST_NONFINITE, I.op, I.node);
          conv = true;
        } else if (err <= P.tol || !(bnext > 0.0)) {
          conv = true;
        }
        pc.lap(P.ctl, 4);
        if (conv || m == mmax) break;
      }
    }
    total_m += m;
    double s_done = s_rem;
    if (!conv && m < N) {
      for (int k = 0; k < 30; ++k) {
        s_done *= 0.5;
        if (threadIdx.x < 32) texp_warp(ks.alpha, ks.beta, m, s_done, ks.ure, ks.uim);
        __syncthreads();
        const double um = sqrt(ks.ure[m - 1] * ks.ure[m - 1] + ks.uim[m - 1] * ks.uim[m - 1]);
        __syncthreads();
        if (bnext * um <= P.tol) break;
      }
      pc.lap(P.ctl, 4);
    }
    // y = beta0 sum_k u_k q_k into the own slice of K_0
    double ny[1] = {0.0};
    for (long long e = e0 + threadIdx.x; e < e1; e += NT) {
      double yr = 0.0, yi = 0.0;
      for (int k = 0; k < m; ++k) {
        const double2 q = Ks(k)[e - e0];
        const double sc = beta0 * ks.scale[k];
        const double cr = ks.ure[k] * sc, ci = ks.uim[k] * sc;
        yr = fma(cr, q.x, fma(-ci, q.y, yr));
        yi = fma(cr, q.y, fma(ci, q.x, yi));
      }
      Ks(0)[e - e0] = make_double2(yr, yi);
      ny[0] = fma(yr, yr, fma(yi, yi, ny[0]));
    }
    if (P.precision != 0) {
      team_allreduce(tm, ny, 1);
      const double ratio = ny[0] > 0.0 ? beta0 / sqrt(ny[0]) : 1.0;
      if (fabs(ratio - 1.0) < 1e-3)
        for (long long e = e0 + threadIdx.x; e < e1; e += NT) {
          const double2 y = Ks(0)[e - e0];
          Ks(0)[e - e0] = make_double2(y.x * ratio, y.y * ratio);
        }
    }
    __syncthreads();
    pc.lap(P.ctl, 5);
    if (conv || m >= N || s_done == s_rem) break;
    s_rem -= s_done;
    if (chunk == 63 && tm.rank == 0 && threadIdx.x == 0) {
      // 64 Krylov spaces did not cover the time step: the result is incomplete
      atomicAdd(&P.ctl->not_converged, 1ull);
      set_status(P.ctl, ST_NOT_CONVERGED, I.op, I.node);
    }
  }
  for (long long e = e0 + threadIdx.x; e < e1; e += NT) x[e] = Ks(0)[e - e0];
  if (tm.rank == 0 && threadIdx.x == 0) {
    P.mhist[I.hist] = m;
    atomicAdd(&P.ctl->krylov_iters, (unsigned long long)total_m);
    atomicAdd(&P.ctl->applies, (unsigned long long)total_m);
    atomicAdd(&P.ctl->flops, I.flops * total_m);
  }
  team_sync(tm);
  return true;
}

// Tiled apply for grid-team nodes too large for shared memory.  The node (legs 0..nl-1, the
// last one physical) is covered twice by tiles:
//   pass A: tiles over legs h..nl-1 (contiguous blocks), one per index of legs 0..h-1;
//   pass B: tiles over legs 0..h-1 and nl-1, one per index of legs h..nl-2;
// with h = (nl - 1) / 2.  A term is computed in the pass whose tile holds all its legs, from
// the tile of the input vector staged in shared memory (every element of a tile is read by
// D of its neighbours along a leg: this replaces strided L2 reads).  Pass A writes its sum,
// pass B adds its terms to it.  Two-stage terms, or a term with legs in neither tile, keep
// the element-wise apply.
struct TiledApply {
  NodeDesc ta, tb;                  // the tile tensors of the two passes
  int h;
  int lmapA[TTNS_MAX_LEGS], lmapB[TTNS_MAX_LEGS];  // tile leg of each node leg (-1: none)
  int nst[TTNS_MAX_LEGS];           // node strides of the tile-B legs 0..h-1
  int bdims[TTNS_MAX_LEGS], bst[TTNS_MAX_LEGS];    // legs h..nl-2: dims and node strides
  int nb;                           // number of such legs
  int nta, ntb;
  unsigned long long inB;           // bit t: term t is computed in pass B
  int ok;
};
__shared__ TiledApply s_tp;

__device__ void tiled_plan(const NodeDesc& nd, const OpStage& os, const TermList& L, TiledApply& tp) {
  const int nl = nd.nl, h = (nl - 1) / 2;
  tp.ok = nl >= 3 && h >= 1 && L.n2 == 0 && L.count <= 64;
  if (!tp.ok) return;
  tp.h = h;
  NodeDesc& a = tp.ta;
  a.nl = nl - h;
  for (int q = 0; q < a.nl; ++q) {
    a.dims[q] = nd.dims[h + q];
    a.strides[q] = nd.strides[h + q];
  }
  a.size = nd.strides[h - 1];
  NodeDesc& b = tp.tb;
  b.nl = h + 1;
  for (int q = 0; q < h; ++q) b.dims[q] = nd.dims[q];
  b.dims[h] = nd.dims[nl - 1];
  b.strides[h] = 1;
  for (int q = h - 1; q >= 0; --q) b.strides[q] = b.strides[q + 1] * b.dims[q + 1];
  b.size = b.strides[0] * b.dims[0];
  for (int q = 0; q < a.nl; ++q) {
    a.inv_dims[q] = 1.0f / (float)a.dims[q];
    a.inv_strides[q] = 1.0f / (float)a.strides[q];
  }
  for (int q = 0; q < b.nl; ++q) {
    b.inv_dims[q] = 1.0f / (float)b.dims[q];
    b.inv_strides[q] = 1.0f / (float)b.strides[q];
  }
  for (int l = 0; l < TTNS_MAX_LEGS; ++l) {
    tp.lmapA[l] = (l >= h && l < nl) ? l - h : -1;
    tp.lmapB[l] = l < h ? l : (l == nl - 1 ? h : -1);
  }
  for (int q = 0; q < h; ++q) tp.nst[q] = nd.strides[q];
  tp.nb = nl - 1 - h;
  for (int q = 0; q < tp.nb; ++q) {
    tp.bdims[q] = nd.dims[h + q];
    tp.bst[q] = nd.strides[h + q];
  }
  tp.nta = (int)(nd.size / a.size);
  tp.ntb = (int)(nd.size / b.size);
  tp.inB = 0ull;
  for (int t = 0; t < L.count; ++t) {
    const Term& tt = os.terms[t];
    bool allA = true, allB = true;
    for (int k = 0; k < tt.nf; ++k) {
      allA = allA && tp.lmapA[tt.f[k].leg] >= 0;
      allB = allB && tp.lmapB[tt.f[k].leg] >= 0;
    }
    if (!allA) {
      if (allB) tp.inB |= 1ull << t;
      else tp.ok = 0;
    }
  }
}

// One pass over this CTA's tiles; emit(global index, sum of the pass's terms at it).
template <typename T, typename F>
__device__ void tiled_pass(const KernelParams& P, Team& tm, const TiledApply& tp, const OpStage& os,
                           const TermList& L, const typename C2<T>::t* xin, typename C2<T>::t* xt, int pass,
                           F&& emit) {
  using V = typename C2<T>::t;
  const NodeDesc& td = pass ? tp.tb : tp.ta;
  const int* lmap = pass ? tp.lmapB : tp.lmapA;
  const int ntiles = pass ? tp.ntb : tp.nta;
  const int TT = td.size;
  const int h = tp.h;
  auto gidx = [&](long long base, int e) -> long long {
    if (!pass) return base + e;
    long long g = base;
    int rem = e;
    for (int q = 0; q < h; ++q) {
      const int iq = fdivu(rem, td.strides[q], td.inv_strides[q]);
      rem -= iq * td.strides[q];
      g += (long long)iq * tp.nst[q];
    }
    return g + rem;  // the physical leg has node stride 1
  };
  for (int tile = tm.rank; tile < ntiles; tile += tm.size) {
    long long base;
    if (!pass) {
      base = (long long)tile * TT;
    } else {
      base = 0;
      int rem = tile;
      for (int q = tp.nb - 1; q >= 0; --q) {
        const int iq = rem % tp.bdims[q];
        rem /= tp.bdims[q];
        base += (long long)iq * tp.bst[q];
      }
    }
    __syncthreads();  // the previous tile's reads are done
    for (int e = threadIdx.x; e < TT; e += NT) xt[e] = xin[gidx(base, e)];
    __syncthreads();
    for (int e = threadIdx.x; e < TT; e += NT) {
      V acc;
      acc.x = acc.y = (T)0;
      for (int t = 0; t < L.count; ++t) {
        if ((int)((tp.inB >> t) & 1ull) != pass) continue;
        Term tt = os.terms[t];
        tt.f[0].leg = lmap[tt.f[0].leg];
        if (tt.nf == 2) tt.f[1].leg = lmap[tt.f[1].leg];
        const V a = tt.nf == 1 ? factor_dot<T>(P, td, tt.f[0], os, xt, e) : direct_dot<T>(P, td, tt, os, xt, e);
        acc.x += a.x;
        acc.y += a.y;
      }
      emit(gidx(base, e), acc);
    }
  }
}

// ------------------------------------------------------------------ tensor-core apply
// H_eff v for a node whose terms have at most one dense factor each (no dense x dense term):
// the terms are grouped by the leg l their dense factor acts on, and every group is one complex
// GEMM on the tensor cores,
//   Y_l[r][i] = sum_{t in group, k} z_t[r][k] M_t[i][k],
// with rows r = the node index with leg l removed, k the index of leg l, z_t = x with the
// term's row-sparse factor (a, a^+, a diagonal or sparse pattern on another leg) applied while
// the operand is staged, and M_t the term's dense matrix (an environment block or a dense
// constant operator).  A task is one group and one tile of 128 rows; K is taken in chunks of at
// most 32 complex values (64 real), so any leg dimension up to 64 fits the shared memory.  The
// result of group g goes to its own compute-type buffer; the terms outside every group (a
// row-sparse factor alone, or a dense factor on a leg below 8) stay on the SIMT path in the pass
// that sums the groups (tc_sum_at).
struct TcPlan {
  int ok;
  int ngroups;
  int gleg[TTNS_MAX_LEGS];
  int gfirst[TTNS_MAX_LEGS + 1];   // terms of group g: gterm[gfirst[g] .. gfirst[g + 1])
  int gterm[TTNS_MAX_TERMS];
  int gdense[TTNS_MAX_TERMS];      // index of the dense factor of each grouped term
  int nsimt;
  int simt[TTNS_MAX_TERMS];        // terms evaluated element-wise
  int gtask0[TTNS_MAX_LEGS + 1];   // first task of group g (tasks of g: K parts x row tiles)
  int gtiles[TTNS_MAX_LEGS];       // row tiles of group g
  int gkpart[TTNS_MAX_LEGS];       // complex K per part (whole chunks)
  int gslot0[TTNS_MAX_LEGS + 1];   // first result slot of group g (one slot per K part)
  float inv_st[TTNS_MAX_LEGS];
};
__shared__ TcPlan s_tcp;

struct TcState {
  uint64_t mbar;
  uint32_t tmem;
  uint32_t phase;
  int on;
};
__shared__ TcState s_tc;

constexpr int kTcRows = 128;   // rows per task (the MMA's M)
constexpr int kTcTmemCols = 512;  // all of an SM's tensor memory (one CTA per SM)
constexpr int kTcSlots = 16;      // compute-type result vectors in the workspace

// Groups, and each group's K (term, leg index) split into parts of whole chunks, one result
// slot per part, so that the tasks (group, part, row tile) run on more CTAs and each runs
// fewer chunks one after another.  ksc: complex K per MMA K step of the precision in use.
__device__ void tc_plan(const NodeDesc& nd, const OpStage& os, const TermList& L, int ksc, TcPlan& tp) {
  tp.ok = 0;
  if (L.n2 > 0 || L.count > TTNS_MAX_TERMS) return;
  int dleg[TTNS_MAX_TERMS], dfac[TTNS_MAX_TERMS];
  for (int t = 0; t < L.count; ++t) {
    const Term& T = os.terms[t];
    dleg[t] = -1;
    dfac[t] = -1;
    if (T.nf == 1) {
      if (T.f[0].nnz == 0 && nd.dims[T.f[0].leg] >= 8) { dleg[t] = T.f[0].leg; dfac[t] = 0; }
    } else if (T.sparse_f >= 0) {
      const int d = 1 - T.sparse_f;
      if (T.f[d].nnz == 0 && nd.dims[T.f[d].leg] >= 8) { dleg[t] = T.f[d].leg; dfac[t] = d; }
    }
  }
  tp.ngroups = 0;
  tp.nsimt = 0;
  int nt = 0;
  for (int l = 0; l < nd.nl; ++l) {
    int c = 0;
    for (int t = 0; t < L.count; ++t) c += dleg[t] == l;
    if (c == 0) continue;
    const int g = tp.ngroups++;
    tp.gleg[g] = l;
    tp.gfirst[g] = nt;
    tp.inv_st[g] = 1.0f / (float)nd.strides[l];
    for (int t = 0; t < L.count; ++t)
      if (dleg[t] == l) { tp.gterm[nt] = t; tp.gdense[nt] = dfac[t]; ++nt; }
  }
  tp.gfirst[tp.ngroups] = nt;
  int ntask = 0, nslot = 0;
  const int cap = tp.ngroups > 0 ? max(1, kTcSlots / tp.ngroups) : 1;
  for (int g = 0; g < tp.ngroups; ++g) {
    const int D = nd.dims[tp.gleg[g]];
    const int Npad = ((2 * D + 15) / 16) * 16;
    const int chunk_kc = min(8, kTcTmemCols / Npad) * ksc;
    const int nterm = tp.gfirst[g + 1] - tp.gfirst[g];
    const int ktot = ((nterm * D + ksc - 1) / ksc) * ksc;
    const int nchunk = (ktot + chunk_kc - 1) / chunk_kc;
    int parts = min(nchunk, cap);
    const int cpp = (nchunk + parts - 1) / parts;  // chunks per part
    parts = (nchunk + cpp - 1) / cpp;
    tp.gkpart[g] = cpp * chunk_kc;
    tp.gtiles[g] = (nd.size / D + kTcRows - 1) / kTcRows;
    tp.gtask0[g] = ntask;
    tp.gslot0[g] = nslot;
    ntask += parts * tp.gtiles[g];
    nslot += parts;
  }
  tp.gtask0[tp.ngroups] = ntask;
  tp.gslot0[tp.ngroups] = nslot;
  for (int t = 0; t < L.count; ++t)
    if (dleg[t] < 0) tp.simt[tp.nsimt++] = t;
  tp.ok = tp.ngroups > 0;
}

// value of z = (row-sparse factor fs, if any) x at idx, in the compute type
template <typename T, typename XT>
__device__ __forceinline__ typename C2<T>::t tc_z(const KernelParams& P, const NodeDesc& nd, const Factor* fs,
                                                  const XT* x, long long idx) {
  if (!fs) return cvt<T>(x[idx]);
  using V = typename C2<T>::t;
  const LegPos lp = leg_pos(nd, fs->leg, idx);
  const int D = nd.dims[fs->leg];
  const V* vals = ops<T>(P) + fs->sp + (long long)lp.i * fs->nnz;
  const V* cols = ops<T>(P) + fs->sp + (long long)D * fs->nnz + (long long)lp.i * fs->nnz;
  V acc;
  acc.x = acc.y = (T)0;
  for (int e = 0; e < fs->nnz; ++e) {
    const int k = (int)cols[e].x;
    cmac<T>(acc, vals[e], cvt<T>(x[lp.base + (long long)k * nd.strides[fs->leg]]));
  }
  return acc;
}

// One task (group g, row tile rt).  K runs over (term, leg index) of the group's terms back to
// back; it is staged in chunks of n_acc MMA K steps, every K step accumulates into its own TMEM
// columns (the tensor core's accumulation rounds toward zero, so a long accumulation drifts),
// and the steps are summed in shared memory in FP32 round-to-nearest, in a fixed order.  The
// operand loads of a thread are issued together (four items at a time) before any is
// converted, so their latencies overlap.  Returns false if a completion wait gave up (the
// status word is set).
template <int KIND, typename T, typename XT>
__device__ __noinline__ bool tc_task(const KernelParams& P, const NodeDesc& nd, const OpStage& os, const TcPlan& tp, int g,
                        int part, int rt, const XT* x, typename C2<T>::t* yg, bool prof) {
  PhaseClock pc;  // phases 20-23 (grid counters): operand staging, MMA completion, read-back, write
  pc.start(prof && threadIdx.x == 0, true);
  using S = tc::Split<KIND>;
  using V = typename C2<T>::t;
  TcState& ts = s_tc;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int l = tp.gleg[g];
  const int D = nd.dims[l];
  const int st = nd.strides[l];
  const int rows = nd.size / D;
  const int r0 = rt * kTcRows;
  const int Npad = ((2 * D + 15) / 16) * 16;
  const int nterm = tp.gfirst[g + 1] - tp.gfirst[g];
  constexpr int G = 8 / S::esize;                // complex values per 16-byte core row
  constexpr int KSC = S::kstep / 2;              // complex K per MMA K step
  const int n_acc = min(8, kTcTmemCols / Npad);   // K steps per chunk, one TMEM slot each
  const int chunk_kc = n_acc * KSC;
  const int ktot = ((nterm * D + KSC - 1) / KSC) * KSC;
  const int ldsum = Npad + 1;
  float* sums = reinterpret_cast<float*>(dyn_smem);
  const uint32_t a_plane = (uint32_t)kTcRows * 2 * chunk_kc * S::esize;
  const uint32_t b_plane = (uint32_t)Npad * 2 * chunk_kc * S::esize;
  const uint32_t sum_bytes = ((uint32_t)kTcRows * ldsum * 4u + 1023u) & ~1023u;
  unsigned char* A = dyn_smem + sum_bytes;
  unsigned char* B = A + S::parts * a_plane;
  // this thread's share of the accumulator: row (TMEM lane) and half of the columns
  const int q4 = warp & 3, half = warp >> 2;
  const int my_row = q4 * 32 + lane;
  const int c_lo = half * (Npad / 2), c_hi = c_lo + Npad / 2;
  for (int c = c_lo; c < c_hi; ++c) sums[my_row * ldsum + c] = 0.0f;
  // Sparse factors with one entry per row (a, a^+, a diagonal): their tables go to shared
  // memory after the operand planes, so that every z of a batch is one independent load of x
  // (else each z would chain a table load and an x load).  Other groups keep tc_z.
  struct SpHdr {
    int sp, leg, st, D;
    float inv_st, inv_D;
    int off, pad;
  };
  unsigned char* tail = B + S::parts * b_plane;
  SpHdr* hdr = reinterpret_cast<SpHdr*>(tail);
  const long long tail_off = (long long)(tail - dyn_smem);
  bool fast = nterm <= TTNS_MAX_TERMS;
  int ntab = 0;
  for (int tl = 0; tl < nterm && fast; ++tl) {
    const int q = tp.gfirst[g] + tl;
    const Term& T_ = os.terms[tp.gterm[q]];
    if (T_.nf == 2) {
      const Factor& f = T_.f[1 - tp.gdense[q]];
      if (f.nnz != 1) fast = false;
      ntab += nd.dims[f.leg];
    }
  }
  const long long hdr_bytes = ((long long)nterm * sizeof(SpHdr) + 15) & ~15LL;
  float2* tvals = reinterpret_cast<float2*>(tail + hdr_bytes);
  int* tcols = reinterpret_cast<int*>(tvals + ntab);
  fast = fast && tail_off + hdr_bytes + (long long)ntab * 12 <= P.smem_bytes;
  if (fast) {
    int off = 0;
    for (int tl = 0; tl < nterm; ++tl) {  // every thread walks the same terms
      const int q = tp.gfirst[g] + tl;
      const Term& T_ = os.terms[tp.gterm[q]];
      SpHdr h{};
      if (T_.nf == 2) {
        const Factor& f = T_.f[1 - tp.gdense[q]];
        h.sp = 1;
        h.leg = f.leg;
        h.st = nd.strides[f.leg];
        h.D = nd.dims[f.leg];
        h.inv_st = nd.inv_strides[f.leg];
        h.inv_D = nd.inv_dims[f.leg];
        h.off = off;
        for (int i = tid; i < h.D; i += NT) {
          tvals[off + i] = P.pool32[f.sp + i];
          tcols[off + i] = (int)P.pool32[f.sp + h.D + i].x;
        }
        off += h.D;
      }
      if (tid == 0) hdr[tl] = h;
    }
    __syncthreads();
  }
  bool ok = true;
  const int kbeg = part * tp.gkpart[g];
  const int kend = min(ktot, kbeg + tp.gkpart[g]);
  for (int kc0 = kbeg; kc0 < kend && ok; kc0 += chunk_kc) {
    const int nk = min(chunk_kc, kend - kc0);   // a multiple of KSC
    const int Kr = 2 * nk;
    // A: rows of the tile x (term, k) of the chunk
    if (fast) {
      const int per_row = nk / G;
      const int nitems = kTcRows * per_row;
      for (int it0 = tid; it0 < nitems; it0 += 4 * NT) {
        long long xi[4][G];
        V cv[4][G];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int item = it0 + u * NT;
          const int row = item % kTcRows, kq = item / kTcRows;
          const int R = r0 + row;
          const bool in = item < nitems && R < rows;
          long long base = 0;
          if (in) {
            const int outer = fdivu(R, st, tp.inv_st[g]);
            base = (long long)outer * D * st + (R - outer * st);
          }
#pragma unroll
          for (int j = 0; j < G; ++j) {
            const int kg = kc0 + kq * G + j;
            xi[u][j] = -1;
            cv[u][j].x = (T)1;
            cv[u][j].y = (T)0;
            if (in && kg < nterm * D) {
              const int tl = kg / D, kk = kg - tl * D;
              const int el = (int)(base + (long long)kk * st);
              const SpHdr h = hdr[tl];
              if (h.sp) {
                const int qq = fdivu(el, h.st, h.inv_st);
                const int i = qq - fdivu(qq, h.D, h.inv_D) * h.D;
                xi[u][j] = (long long)(el - i * h.st) + (long long)tcols[h.off + i] * h.st;
                const float2 v = tvals[h.off + i];
                cv[u][j].x = (T)v.x;
                cv[u][j].y = (T)v.y;
              } else {
                xi[u][j] = el;
              }
            }
          }
        }
        V xv[4][G];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int j = 0; j < G; ++j) {
            if (xi[u][j] >= 0) {
              xv[u][j] = cvt<T>(x[xi[u][j]]);
            } else {
              xv[u][j].x = (T)0;
              xv[u][j].y = (T)0;
            }
          }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int item = it0 + u * NT;
          if (item >= nitems) break;
          const int row = item % kTcRows, kq = item / kTcRows;
#pragma unroll
          for (int j = 0; j < G; ++j) {
            V z;
            z.x = z.y = (T)0;
            cmac<T>(z, cv[u][j], xv[u][j]);
            tc::put_split_f<KIND>(A, a_plane, row, 2 * (kq * G + j), Kr, (float)z.x);
            tc::put_split_f<KIND>(A, a_plane, row, 2 * (kq * G + j) + 1, Kr, (float)z.y);
          }
        }
      }
    } else {
      const int per_row = nk / G;
      const int nitems = kTcRows * per_row;
      for (int it0 = tid; it0 < nitems; it0 += 4 * NT) {
        float re[4][G], im[4][G];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int item = it0 + u * NT;
          const int row = item % kTcRows, kq = item / kTcRows;
          const int R = r0 + row;
          const bool in = item < nitems && R < rows;
          long long base = 0;
          if (in) {
            const int outer = fdivu(R, st, tp.inv_st[g]);
            base = (long long)outer * D * st + (R - outer * st);
          }
#pragma unroll
          for (int j = 0; j < G; ++j) {
            const int kg = kc0 + kq * G + j;   // global K index: term kg / D, leg index kg % D
            V z;
            z.x = z.y = (T)0;
            if (in && kg < nterm * D) {
              const int tl = kg / D, kk = kg - tl * D;
              const int q = tp.gfirst[g] + tl;
              const Term& T_ = os.terms[tp.gterm[q]];
              const Factor* fs = T_.nf == 2 ? &T_.f[1 - tp.gdense[q]] : nullptr;
              z = tc_z<T>(P, nd, fs, x, base + (long long)kk * st);
            }
            re[u][j] = (float)z.x;
            im[u][j] = (float)z.y;
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int item = it0 + u * NT;
          if (item >= nitems) break;
          const int row = item % kTcRows, kq = item / kTcRows;
#pragma unroll
          for (int j = 0; j < G; ++j) {
            tc::put_split_f<KIND>(A, a_plane, row, 2 * (kq * G + j), Kr, re[u][j]);
            tc::put_split_f<KIND>(A, a_plane, row, 2 * (kq * G + j) + 1, Kr, im[u][j]);
          }
        }
      }
    }
    // B: the 2 x 2 real blocks of M_t[i][k]: rows 2i (a, -b) and 2i + 1 (b, a)
    {
      const int per_i = nk / G;
      const int nitems = (Npad / 2) * per_i;
      for (int item = tid; item < nitems; item += NT) {
        const int kq = item % per_i, i = item / per_i;
        float2 m[G];
#pragma unroll
        for (int j = 0; j < G; ++j) {
          const int kg = kc0 + kq * G + j;
          m[j] = make_float2(0.f, 0.f);
          if (i < D && kg < nterm * D) {
            const int tl = kg / D, kk = kg - tl * D;
            const int q = tp.gfirst[g] + tl;
            const Factor& fd = os.terms[tp.gterm[q]].f[tp.gdense[q]];
            m[j] = P.pool32[fd.mat + (long long)i * D + kk];
          }
        }
#pragma unroll
        for (int j = 0; j < G; ++j) {
          const int k = kq * G + j;
          tc::put_split_f<KIND>(B, b_plane, 2 * i, 2 * k, Kr, m[j].x);
          tc::put_split_f<KIND>(B, b_plane, 2 * i, 2 * k + 1, Kr, -m[j].y);
          tc::put_split_f<KIND>(B, b_plane, 2 * i + 1, 2 * k, Kr, m[j].y);
          tc::put_split_f<KIND>(B, b_plane, 2 * i + 1, 2 * k + 1, Kr, m[j].x);
        }
      }
    }
    tc::fence_proxy_async();
    __syncthreads();
    pc.lap(P.ctl, 20);
    const int nsteps = nk / KSC;
    if (tid == 0) {
      tc::fence_after();
      for (int ks = 0; ks < nsteps; ++ks)
        tc::issue_kstep<KIND>(ts.tmem + (uint32_t)(ks * Npad), A, a_plane, B, b_plane, Npad, Kr, ks);
      tc::commit(&ts.mbar);
    }
    const bool w = tc::mbar_wait(&ts.mbar, ts.phase, P.spin_limit);
    tc::fence_after();
    ok = __syncthreads_and(w) != 0;  // the same decision on every thread
    if (!ok) break;
    if (tid == 0) ts.phase ^= 1u;
    pc.lap(P.ctl, 21);
    // the K steps' partial products, summed in a fixed order into the shared FP32 sums; the
    // loads of all K steps of a column group are issued before one wait
    const uint32_t lane_base = ts.tmem + ((uint32_t)(q4 * 32) << 16);
    for (int c = c_lo; c < c_hi; c += 8) {
      uint32_t r[8][8];
#pragma unroll
      for (int ks = 0; ks < 8; ++ks)
        if (ks < nsteps) tc::tmem_ld8_nowait(lane_base + (uint32_t)(ks * Npad + c), r[ks]);
      tc::tmem_wait_ld();
      float acc[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] = 0.0f;
#pragma unroll
      for (int ks = 0; ks < 8; ++ks)
        if (ks < nsteps) {
          tc::tmem_pin8(r[ks]);
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[j] += __uint_as_float(r[ks][j]);
        }
#pragma unroll
      for (int j = 0; j < 8; ++j) sums[my_row * ldsum + c + j] += acc[j];
    }
    tc::fence_before();
    __syncthreads();
    pc.lap(P.ctl, 22);
  }
  if (!ok) {
    // a completion wait gave up: report it, give the MMAs in flight a last bounded wait, and
    // leave the tensor cores alone in this CTA for the rest of the launch
    if (tid == 0) set_status(P.ctl, ST_TIMEOUT, 400, -1);
    tc::mbar_wait(&ts.mbar, ts.phase, P.spin_limit);
    __syncthreads();
    if (tid == 0) ts.on = 0;
    __syncthreads();
    return false;
  }
  // the tile's rows of Y_g: row R = (outer, inner) of leg l, column pair (2i, 2i + 1) = y[.., i, ..]
  const int R = r0 + my_row;
  if (R < rows) {
    const int outer = fdivu(R, st, tp.inv_st[g]);
    const long long base = (long long)outer * D * st + (R - outer * st);
    for (int c = c_lo; c < c_hi; c += 2) {
      const int i = c >> 1;
      if (i < D) {
        V y;
        y.x = (T)sums[my_row * ldsum + c];
        y.y = (T)sums[my_row * ldsum + c + 1];
        yg[base + (long long)i * st] = y;
      }
    }
  }
  __syncthreads();
  pc.lap(P.ctl, 23);
  return true;
}

// All tasks of the plan over the team's CTAs (task k on rank k mod size).  The result of
// part p of group g goes to slot gslot0[g] + p at ybuf + slot * ystride.  The caller
// synchronises the team before reading the slots.
template <typename T, typename XT>
__device__ void tc_apply(const KernelParams& P, Team& tm, const NodeDesc& nd, const OpStage& os, const TcPlan& tp,
                         const XT* x, typename C2<T>::t* ybuf, long long ystride) {
  const int ntask = tp.gtask0[tp.ngroups];
  for (int task = tm.rank; task < ntask; task += tm.size) {
    int g = 0;
    while (task >= tp.gtask0[g + 1]) ++g;
    const int local = task - tp.gtask0[g];
    const int part = local / tp.gtiles[g], rt = local - part * tp.gtiles[g];
    auto* yg = ybuf + (long long)(tp.gslot0[g] + part) * ystride;
    const bool prof = P.profile && tm.rank == 0;
    const bool ok = P.precision == 2 ? tc_task<tc::KIND_BF16X3, T>(P, nd, os, tp, g, part, rt, x, yg, prof)
                                     : tc_task<tc::KIND_TF32X3, T>(P, nd, os, tp, g, part, rt, x, yg, prof);
    if (!ok) break;
  }
}

// H_eff x at idx from the group results and the terms left to the SIMT path
template <typename T, typename XT>
__device__ __forceinline__ typename C2<T>::t tc_sum_at(const KernelParams& P, const NodeDesc& nd, const OpStage& os,
                                                      const TcPlan& tp, const XT* x,
                                                      const typename C2<T>::t* ybuf, long long ystride,
                                                      long long idx) {
  typename C2<T>::t acc;
  acc.x = acc.y = (T)0;
  const int nslot = tp.gslot0[tp.ngroups];
  for (int sl = 0; sl < nslot; ++sl) {
    const auto y = ybuf[sl * ystride + idx];
    acc.x += y.x;
    acc.y += y.y;
  }
  for (int q = 0; q < tp.nsimt; ++q) {
    const Term& T_ = os.terms[tp.simt[q]];
    const auto a = T_.nf == 1 ? factor_dot<T>(P, nd, T_.f[0], os, x, idx) : direct_dot<T>(P, nd, T_, os, x, idx);
    acc.x += a.x;
    acc.y += a.y;
  }
  return acc;
}

template <typename T>
__device__ __noinline__ void op_expm(const KernelParams& P, Team& tm, const Instr& I, double2* work, double tau) {
  KrylovShared& ks = s_ks;
  PhaseClock pc;
  pc.start(P.profile && tm.rank == 0 && threadIdx.x == 0, tm.kind == TEAM_GRID);
  const NodeDesc nd = P.nodes[I.node];
  const TermList L = P.lists[I.terms];
  const long long N = nd.size;
  const long long kv = P.kvec;
  double2* x = P.pool + nd.off;
  double2* Kb = work;                           // K_1..K_mmax at Kb + (j-1)*kv
  auto* tmp = reinterpret_cast<typename C2<T>::t*>(work + (long long)P.mmax * kv);  // n_tmp temporaries
  auto Kp = [&](int j) -> double2* { return j == 0 ? x : Kb + (long long)(j - 1) * kv; };
  const int mmax = min(P.mmax, (int)(N < (long long)TTNS_KMAX ? N : (long long)TTNS_KMAX));
  OpStage& os = s_os;
  stage_op<T>(P, I, L, nullptr, 0, os);
  using V = typename C2<T>::t;
  // tensor-core apply (split precision) for nodes whose terms have one dense factor each; its
  // operand tiles take the dynamic shared memory, so nothing staged there is used
  bool use_tc = false;
  if (s_tc.on && (P.precision == 1 || P.precision == 2) && N >= 4096) {
    if (threadIdx.x == 0) {
      tc_plan(nd, os, L, P.precision == 2 ? tc::Split<tc::KIND_BF16X3>::kstep / 2 : tc::Split<tc::KIND_TF32X3>::kstep / 2,
              s_tcp);
      if (s_tcp.ok) {
        os.a_n = os.b_n = 0;
        os.end = 0;
      }
    }
    __syncthreads();
    use_tc = s_tcp.ok != 0;
  }
  V* ybuf = reinterpret_cast<V*>(work + (long long)(P.mmax + P.n_tmp + 2) * kv);  // group results (TC)
  V* xs = use_tc ? nullptr : vec_smem<T>(P, os, N);  // input vector in shared memory when it fits
  // otherwise, in mixed precision, a compute-type copy of the input vector in the workspace,
  // written by the pass that produces the vector (FP64 Krylov basis, FP32 operand)
  // (kept in the mixed modes whether or not the vector is staged: staging then copies it
  // instead of converting the FP64 vector on every CTA)
  constexpr bool kShadow = !std::is_same<T, double>::value;
  V* xf = reinterpret_cast<V*>(work + (long long)(P.mmax + P.n_tmp) * kv);
  const bool shadow = kShadow;
  // tiled apply for a grid-team node that does not fit in shared memory
  TiledApply& tp = s_tp;
  V* xt = nullptr;
  bool tiled = false;
  if (tm.kind == TEAM_GRID && xs == nullptr && !use_tc) {
    if (threadIdx.x == 0) tiled_plan(nd, os, L, tp);
    __syncthreads();
    if (tp.ok) {
      xt = vec_smem<T>(P, os, tp.ta.size > tp.tb.size ? tp.ta.size : tp.tb.size);
      tiled = xt != nullptr;  // the same on every CTA
    }
  }
  pc.lap(P.ctl, 0);
  // exp(-i s H): s = time / hbar with the op's sign.  If the Krylov space of dimension
  // mmax does not reach the tolerance for the remaining time, the largest s / 2^k that
  // does is taken on the same space and a new space is built for the rest.
  double s_rem = I.sign * tau / HBAR_EVFS;
  int total_m = 0;
  int m = 0;
  for (int chunk = 0; chunk < 64; ++chunk) {
    double v[1];
    v[0] = 0;
    for (long long idx = tm.gtid(); idx < N; idx += tm.nthr()) {
      const double2 a = x[idx];
      v[0] = fma(a.x, a.x, fma(a.y, a.y, v[0]));
      if (shadow) xf[idx] = cvt<T>(a);
    }
    team_allreduce(tm, v, 1);
    const double beta0 = sqrt(v[0]);
    pc.lap(P.ctl, 6);
    if (!(beta0 > 0.0)) {
      if (!(beta0 == 0.0)) set_status(P.ctl, ST_NONFINITE, I.op, I.node);
      break;
    }
    if (threadIdx.x == 0) {
      ks.scale[0] = 1.0 / beta0;
      ks.beta[0] = 0.0;
    }
    __syncthreads();
    m = 0;
    bool conv = false;
    double bnext = 0.0;
    // leading-order size of |e_m^T exp(-i s T_m) e_0|: |s|^(m-1) prod beta_i / (m-1)!,
    // used to decide when the exact (small-exponential) check is worth running
    double lead = 1.0;
    int next_check = 1;
    for (int j = 0; j < mmax; ++j) {
      double2* Kj = Kp(j);
      double2* Kjm = j > 0 ? Kp(j - 1) : x;
      double2* W = Kb + (long long)j * kv;  // slot of K_{j+1}
      const double sj = ks.scale[j];
      const double bj = ks.beta[j];
      const double sjm = j > 0 ? ks.scale[j - 1] : 0.0;
      if (xs) {
        if constexpr (kShadow)
          stage_copy(xs, xf, N);
        else
          stage_vector<T>(xs, Kj, N);
      }
      // operand of this application: shared memory, the FP32 shadow, or K_j itself (FP64)
      const V* xin = xs ? xs : (shadow ? xf : reinterpret_cast<const V*>(Kj));
      if (L.n2 > 0) {
        apply_stage1<T>(P, tm, nd, xin, L, tmp, kv, os);
        team_sync(tm);
      }
      pc.lap(P.ctl, 1);
      // part[0] = Re <K_j, w>; in mixed precision also part[1] = |w|^2 (one reduction for
      // alpha_j and beta_{j+1}, as in the cluster-resident form)
      const bool mixed = P.precision != 0;
      double part[3] = {0.0, 0.0, 0.0};
      auto recur = [&](long long idx, V a) {  // w = s_j H K_j - beta_j q_{j-1} at idx, and the dots
        const double2 kj = Kj[idx];
        double wr = sj * (double)a.x, wi = sj * (double)a.y;
        if (j > 0) {
          const double2 km = Kjm[idx];
          wr = fma(-bj * sjm, km.x, wr);
          wi = fma(-bj * sjm, km.y, wi);
        }
        W[idx] = make_double2(wr, wi);
        part[0] = fma(kj.x, wr, fma(kj.y, wi, part[0]));  // Re(conj(K_j) w)
        if (mixed) {
          part[1] = fma(wr, wr, fma(wi, wi, part[1]));
          part[2] = fma(kj.x, kj.x, fma(kj.y, kj.y, part[2]));
        }
      };
      if (use_tc) {
        tc_apply<T>(P, tm, nd, os, s_tcp, xin, ybuf, kv);
        team_sync(tm);
        pc.lap(P.ctl, 7);
        for (long long idx = tm.gtid(); idx < N; idx += tm.nthr())
          recur(idx, tc_sum_at<T>(P, nd, os, s_tcp, xin, ybuf, kv, idx));
      } else if (tiled) {
        V* y = tmp;  // pass A sums (no two-stage terms, so the temporaries are free)
        tiled_pass<T>(P, tm, tp, os, L, xin, xt, 0, [&](long long g, V acc) { y[g] = acc; });
        team_sync(tm);
        tiled_pass<T>(P, tm, tp, os, L, xin, xt, 1, [&](long long g, V acc) {
          V a = y[g];
          a.x += acc.x;
          a.y += acc.y;
          recur(g, a);
        });
      } else {
        for (long long idx = tm.gtid(); idx < N; idx += tm.nthr()) recur(idx, apply_stage2_at<T>(P, nd, xin, L, tmp, kv, idx, os));
      }
      team_allreduce(tm, part, mixed ? 3 : 1);
      pc.lap(P.ctl, 2);
      const double aj = part[0] * sj;
      // |w - alpha_j q_j|^2 = |w|^2 - 2 alpha_j^2 + alpha_j^2 |q_j|^2 with |q_j|^2 from the same
      // reduction (the error of an assumed |q_j| = 1 would grow by alpha^2 / beta^2 per step);
      // used unless it cancels (the same decision on every CTA)
      const double nq = sj * sj * part[2];
      const double b2 = part[1] - aj * aj * (2.0 - nq);
      const bool fused = mixed && b2 > 1e-4 * part[1];
      double nrm[1] = {0.0};
      for (long long idx = tm.gtid(); idx < N; idx += tm.nthr()) {
        const double2 kj = Kj[idx];
        double2 w = W[idx];
        w.x = fma(-aj * sj, kj.x, w.x);
        w.y = fma(-aj * sj, kj.y, w.y);
        W[idx] = w;
        if (shadow) xf[idx] = cvt<T>(w);  // every read of the old shadow ended at the last barrier
        nrm[0] = fma(w.x, w.x, fma(w.y, w.y, nrm[0]));
      }
      if (P.precision == 0) nrm[0] = reorth_strided(tm, N, x, Kb, kv, W, j, ks);
      if (fused) {
        bnext = sqrt(b2);
        team_sync(tm);  // K_{j+1} and its shadow are complete before the next application
      } else {
        team_allreduce(tm, nrm, 1);
        bnext = sqrt(nrm[0]);
      }
      pc.lap(P.ctl, 3);
      if (threadIdx.x == 0) {
        ks.alpha[j] = aj;
        ks.beta[j + 1] = bnext;
        ks.scale[j + 1] = bnext > 0.0 ? 1.0 / bnext : 0.0;
      }
      __syncthreads();
      m = j + 1;
      const double est = bnext * lead;
      lead *= fabs(s_rem) * bnext / (double)m;
      if ((est <= 1e2 * P.tol && m >= next_check) || m == mmax || !(bnext > 0.0)) {
        next_check = m + 1;
        if (threadIdx.x < 32) texp_warp(ks.alpha, ks.beta, m, s_rem, ks.ure, ks.uim);
        __syncthreads();
        const double um = sqrt(ks.ure[m - 1] * ks.ure[m - 1] + ks.uim[m - 1] * ks.uim[m - 1]);
        const double err = bnext * um;
        if (!(err == err)) {
          set_status(P.ctl, ST_NONFINITE, I.op, I.node);
          conv = true;
        } else if (err <= P.tol || !(bnext > 0.0)) {
          conv = true;
        }
        pc.lap(P.ctl, 4);
        if (conv || m == mmax) break;
      }
    }
    total_m += m;
    double s_done = s_rem;
    if (!conv && m < N) {
      // largest s_rem / 2^k that converges on this space (same decision on every CTA)
      for (int k = 0; k < 30; ++k) {
        s_done *= 0.5;
        if (threadIdx.x < 32) texp_warp(ks.alpha, ks.beta, m, s_done, ks.ure, ks.uim);
        __syncthreads();
        const double um = sqrt(ks.ure[m - 1] * ks.ure[m - 1] + ks.uim[m - 1] * ks.uim[m - 1]);
        __syncthreads();
        if (bnext * um <= P.tol) break;
      }
      pc.lap(P.ctl, 4);
    }
    // y = beta0 * sum_k u_k q_k written over x (each thread reads its own K_0 = x entries first)
    double ny[1] = {0.0};
    for (long long idx = tm.gtid(); idx < N; idx += tm.nthr()) {
      double yr = 0.0, yi = 0.0;
      for (int k = 0; k < m; ++k) {
        const double2 q = Kp(k)[idx];
        const double sc = beta0 * ks.scale[k];
        const double cr = ks.ure[k] * sc, ci = ks.uim[k] * sc;
        yr = fma(cr, q.x, fma(-ci, q.y, yr));
        yi = fma(cr, q.y, fma(ci, q.x, yi));
      }
      x[idx] = make_double2(yr, yi);
      ny[0] = fma(yr, yr, fma(yi, yi, ny[0]));
    }
    if (P.precision != 0) {
      // The exact exponential is unitary.  FP32-class contractions leave the Krylov basis
      // orthonormal only to ~1e-7, so the combination's norm is restored to the input's.
      team_allreduce(tm, ny, 1);
      const double ratio = ny[0] > 0.0 ? beta0 / sqrt(ny[0]) : 1.0;
      if (fabs(ratio - 1.0) < 1e-3) {
        for (long long idx = tm.gtid(); idx < N; idx += tm.nthr()) {
          double2 y = x[idx];
          x[idx] = make_double2(y.x * ratio, y.y * ratio);
        }
      }
    }
    team_sync(tm);
    pc.lap(P.ctl, 5);
    if (conv || m >= N || s_done == s_rem) break;
    s_rem -= s_done;
    if (chunk == 63 && tm.rank == 0 && threadIdx.x == 0) {
      // 64 Krylov spaces did not cover the time step: the result is incomplete
      atomicAdd(&P.ctl->not_converged, 1ull);
      set_status(P.ctl, ST_NOT_CONVERGED, I.op, I.node);
    }
  }
  if (tm.rank == 0 && threadIdx.x == 0) {
    P.mhist[I.hist] = m;
    atomicAdd(&P.ctl->krylov_iters, (unsigned long long)total_m);
    atomicAdd(&P.ctl->applies, (unsigned long long)total_m);
    atomicAdd(&P.ctl->flops, I.flops * total_m);
  }
}

// ------------------------------------------------------------------ Householder QR
// A_v (matricised: rows = all other legs in order, columns = leg I.leg) = Q R with the
// completion rule of the oracle: null sub-columns (norm <= qr_cutoff ||M||_F) get the identity
// reflector and R_jj = 0; Q = H_0 ... H_{n-1} I[:, :n] through the compact WY form
// Q = I - V T V^H; finally R_jj is made real and >= 0.  FP64.
struct QRShared {
  double tau[TTNS_MAX_D];    // H_j = I - tau_j v_j v_j^H with the unnormalised v_j of the column loop
  double shat[TTNS_MAX_D];   // 1 / |v_j| = sqrt(tau_j / 2) (0 for an identity reflector)
  double2 coef[TTNS_MAX_D];  // tau_j v_j^H W[k] of the trailing columns
  double2 vhead[TTNS_MAX_D];
  double2 rdiag[TTNS_MAX_D];
  double2 ph[TTNS_MAX_D];
};
__shared__ QRShared s_qs;


__device__ __forceinline__ long long qr_addr(const NodeDesc& nd, int l, long long r, int c) {
  const int st = nd.strides[l];
  const int p = fdivu((int)r, st, nd.inv_strides[l]);
  const int q = (int)r - p * st;
  return (long long)(p * nd.dims[l] * st + c * st + q);
}

// Every CTA of the team owns a contiguous chunk of rows [rb, re); loops inside a CTA run
// over (column, row) pairs so that small chunks (a few rows per CTA) still occupy the
// threads.  The FP64 work is spread over all SMs of the team.
__device__ __noinline__ void op_qr(const KernelParams& P, Team& tm, const Instr& I, double2* work) {
  QRShared& qs = s_qs;
  PhaseClock pc;
  pc.start(P.profile && tm.rank == 0 && threadIdx.x == 0, tm.kind == TEAM_GRID);
  const NodeDesc nd = P.nodes[I.node];
  const int l = I.leg;
  const int n = nd.dims[l];
  const long long rows = nd.size / n;
  double2* A = P.pool + nd.off;
  double2* W = work;  // column-major: W[c * rows + r]
  double2* Rout = P.pool + P.trees[I.tree].bond_off;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long chunk = (rows + tm.size - 1) / tm.size;
  const long long rb = min(rows, (long long)tm.rank * chunk);
  const long long re = min(rows, rb + chunk);
  const int nr = (int)(re - rb);
  const float inv_nr = nr > 0 ? 1.0f / (float)nr : 0.0f;
  // reduction buffers in the dynamic shared memory (no operator is staged during a QR)
  const int PB = max(2 * n * n, 4 * n + 4);
  double* red[2] = {reinterpret_cast<double*>(dyn_smem), reinterpret_cast<double*>(dyn_smem) + PB};
  double* redo = red[1] + PB;
  int rp = 0;
  // the CTA's own rows of the workspace matrix stay in shared memory during the QR when
  // they fit (column-major, `chunk` rows per column); rows < n, which other CTAs read for T,
  // Z and R, are also written to the global workspace after the column loop
  const long long ws_off = (3LL * PB * (long long)sizeof(double) + 15) & ~15LL;
  const bool in_smem = ws_off + (long long)n * chunk * (long long)sizeof(double2) <= P.smem_bytes;
  double2* const Wl = in_smem ? reinterpret_cast<double2*>(dyn_smem + ws_off) : W;
  const long long ldw = in_smem ? chunk : rows;
  const long long roff = in_smem ? rb : 0;
  auto WA = [&](int c, long long r) -> double2& { return Wl[(long long)c * ldw + (r - roff)]; };
  // the small matrices G (Gram of the reflectors), T and Z (n x n, row stride ldg): after the
  // rows in shared memory when they fit there too, else in the per-CTA global scratch
  const long long g_off = (ws_off + (in_smem ? (long long)n * chunk * (long long)sizeof(double2) : 0) + 15) & ~15LL;
  const bool g_smem = g_off + 3LL * n * n * (long long)sizeof(double2) <= P.smem_bytes;
  const int ldg = g_smem ? n : TTNS_MAX_D;
  double2* G = g_smem ? reinterpret_cast<double2*>(dyn_smem + g_off)
                      : P.cta_scratch + (long long)blockIdx.x * P.cta_scratch_stride;
  double2* Tm = G + ldg * ldg;
  double2* Z = Tm + ldg * ldg;
  // copy into the column-major workspace; the Frobenius norm sets the null threshold
  double fro = 0.0;
  for (int idx = threadIdx.x; idx < n * nr; idx += NT) {
    const int c = fdivu(idx, nr, inv_nr);
    const long long r = rb + (idx - c * nr);
    const double2 a = A[qr_addr(nd, l, r, c)];
    WA(c, r) = a;
    fro = fma(a.x, a.x, fma(a.y, a.y, fro));
  }
  __syncthreads();  // copied with the pair mapping, read below per lane
  // One team reduction per column.  Before reflecting column j every CTA needs, over its
  // rows r > j and for the columns c = j .. n-1,
  //   d_c = sum_r conj(W[j][r]) W[c][r]   and   h_c = W[c][j]  (row j: its owner only),
  // in slots [4 (c - j) .. 4 (c - j) + 4).  Then sigma_j^2 = |h_j|^2 + d_j, x0 = h_j, and
  // c_k = tau (d_k + conj(vh) h_k) is v^H W[k] with the head of v replaced by vh.
  // Products and sums are packed so that few FP64 instructions run with idle lanes: when
  // the CTA's rows below jj number at most 32, one thread forms each (column, row) product
  // into shared memory and the per-column sums are fixed trees; for more rows, warps take
  // columns four at a time with a transposing butterfly.
  // product scratch (n x 32 complex) after G, T, Z
  const long long p_off = (g_off + (g_smem ? 3LL * n * n * (long long)sizeof(double2) : 0) + 15) & ~15LL;
  const bool p_smem = g_smem && p_off + 32LL * n * (long long)sizeof(double2) <= P.smem_bytes;
  double2* const prod = reinterpret_cast<double2*>(dyn_smem + p_off);
  auto prepare = [&](int jj, double* mine) {
    const int nc = n - jj;
    const long long r1 = max(rb, (long long)jj + 1);
    const int nrw = (int)max(0LL, re - r1);  // own rows strictly below row jj
    if (p_smem && chunk <= 32) {  // the same branch on every CTA (chunk is uniform)
      // prod[c * 32 + r] = conj(v_r) W[jj + c][r], zero-padded to 32 rows
      for (int idx = threadIdx.x; idx < nc * 32; idx += NT) {
        const int c = idx >> 5, rr = idx & 31;
        double2 p = make_double2(0.0, 0.0);
        if (rr < nrw) {
          const long long r = r1 + rr;
          const double2 vr = WA(jj, r), w = WA(jj + c, r);
          p = make_double2(fma(vr.x, w.x, vr.y * w.y), fma(vr.x, w.y, -vr.y * w.x));
        }
        prod[idx] = p;
      }
      __syncthreads();
      // per column: 8 threads add 4 rows each, then a fixed tree over the 8 partials (the
      // trip count is rounded to whole warps so that every lane takes part in the shuffles)
      const int ntask = nc * 8;
      for (int idx = threadIdx.x; idx < ((ntask + 31) & ~31); idx += NT) {
        const bool on = idx < ntask;
        const int c = idx >> 3, g = idx & 7;
        double sr = 0.0, si = 0.0;
        if (on) {
          const double2* pc2 = prod + c * 32 + g;
          const double2 s0 = pc2[0], s1 = pc2[8], s2 = pc2[16], s3 = pc2[24];
          sr = (s0.x + s1.x) + (s2.x + s3.x);
          si = (s0.y + s1.y) + (s2.y + s3.y);
        }
#pragma unroll
        for (int o = 4; o >= 1; o >>= 1) {  // within the aligned group of 8 lanes
          sr += __shfl_xor_sync(0xffffffffu, sr, o);
          si += __shfl_xor_sync(0xffffffffu, si, o);
        }
        if (on && g == 0) {
          mine[4 * c] = sr;
          mine[4 * c + 1] = si;
        }
      }
    } else {
      for (int c0 = 0; c0 < nc; c0 += 4 * NWARP) {
        double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (long long r = r1 + lane; r < re; r += 32) {
          const double2 vr = WA(jj, r);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int c = c0 + warp + q * NWARP;
            if (c < nc) {
              const double2 w = WA(jj + c, r);
              acc[2 * q] = fma(vr.x, w.x, fma(vr.y, w.y, acc[2 * q]));
              acc[2 * q + 1] = fma(vr.x, w.y, fma(-vr.y, w.x, acc[2 * q + 1]));
            }
          }
        }
        const double t = warp_reduce_t<8>(acc);
        if ((lane & 3) == 0) {
          const int vid = warp_reduce_vid<8>(lane);
          const int c = c0 + warp + (vid >> 1) * NWARP;
          if (c < nc) mine[4 * c + (vid & 1)] = t;
        }
      }
    }
    const bool own_row = rb <= jj && jj < re;
    for (int c = threadIdx.x; c < nc; c += NT) {
      const double2 h = own_row ? WA(jj + c, jj) : make_double2(0.0, 0.0);
      mine[4 * c + 2] = h.x;
      mine[4 * c + 3] = h.y;
    }
  };
  {
    double* mine = red[rp];
    rp ^= 1;
    prepare(0, mine);
    // the Frobenius norm rides along in the first reduction
    __shared__ double s_fro[NWARP];
    const double f = warp_sum(fro);
    if (lane == 0) s_fro[warp] = f;
    __syncthreads();
    if (threadIdx.x == 0) {
      double sum = 0.0;
      for (int w = 0; w < NWARP; ++w) sum += s_fro[w];
      mine[4 * n] = sum;
    }
    team_reduce_vec(tm, mine, redo, 4 * n + 1);
  }
  pc.lap(P.ctl, 8);
  const double fro_m = sqrt(redo[4 * n]);  // ||M||_F (redo is reused by the column loop)
  const double thr = P.qr_cutoff * fro_m;
  for (int j = 0; j < n; ++j) {
    // reflector of column j: alpha = -phase(x0) sigma, vh = x0 - alpha = x0 (1 + sigma / |x0|),
    // |vh| = |x0| + sigma, |v|^2 = d_j + |vh|^2, tau = 2 / |v|^2.  Written so that the FP64
    // square roots and divisions (long dependent sequences on this part) overlap.
    const double2 x0 = make_double2(redo[2], redo[3]);
    const double ax2 = x0.x * x0.x + x0.y * x0.y;
    const double sigma = sqrt(ax2 + redo[0]);
    const double ax = sqrt(ax2);
    double tau = 0.0, shat = 0.0;
    double2 vh = make_double2(0, 0), alpha = make_double2(0, 0);
    const bool null = !(sigma > thr);
    if (!null) {
      // a head below 1e-280 counts as zero (phase 1): its reciprocal would overflow
      const bool head = ax > 1e-280;
      const double inv_ax = head ? 1.0 / ax : 0.0;
      const double hv = ax + sigma;
      const double vn2 = redo[0] + hv * hv;
      tau = 2.0 / vn2;
      shat = rsqrt(vn2);
      if (head) {
        const double f = sigma * inv_ax;
        alpha = make_double2(-f * x0.x, -f * x0.y);
        vh = make_double2(x0.x + f * x0.x, x0.y + f * x0.y);
      } else {
        alpha = make_double2(-sigma, 0.0);
        vh = make_double2(sigma, 0.0);
      }
    }
    const int nk = n - j - 1;
    if (threadIdx.x == 0) {
      qs.tau[j] = tau;
      qs.shat[j] = shat;
      qs.vhead[j] = vh;
      qs.rdiag[j] = alpha;
    }
    if (!null && nk > 0) {
      // c_k = tau (d_k + conj(vh) h_k) for the trailing columns k = j+1 ..
      for (int k = threadIdx.x; k < nk; k += NT) {
        const int sl = 4 * (k + 1);
        const double dr = redo[sl] + (vh.x * redo[sl + 2] + vh.y * redo[sl + 3]);
        const double di = redo[sl + 1] + (vh.x * redo[sl + 3] - vh.y * redo[sl + 2]);
        qs.coef[k] = make_double2(tau * dr, tau * di);
      }
      __syncthreads();
      pc.lap(P.ctl, 13);
      // update the trailing columns on the own rows r >= j
      const long long r0 = max(rb, (long long)j);
      const int nrr = (int)max(0LL, re - r0);
      const float inv_nrr = nrr > 0 ? 1.0f / (float)nrr : 0.0f;
      for (int idx = threadIdx.x; idx < nk * nrr; idx += NT) {
        const int k = fdivu(idx, nrr, inv_nrr);
        const long long r = r0 + (idx - k * nrr);
        const double2 vr = (r == j) ? vh : WA(j, r);
        const double2 ck = qs.coef[k];
        double2* wp = &WA(j + 1 + k, r);
        double2 w = *wp;
        w.x -= vr.x * ck.x - vr.y * ck.y;
        w.y -= vr.x * ck.y + vr.y * ck.x;
        *wp = w;
      }
    }
    if (nk > 0) {
      __syncthreads();  // the updates (pair mapping) before the next column's dots (lane mapping)
      pc.lap(P.ctl, 14);
      double* mine = red[rp];
      rp ^= 1;
      prepare(j + 1, mine);
      pc.lap(P.ctl, 15);
      team_reduce_vec(tm, mine, redo, 4 * nk);
      pc.lap(P.ctl, 9);
    }
  }
  __syncthreads();
  if (in_smem) {  // rows < n to the global workspace (read across CTAs below)
    const long long rt = min(re, (long long)n);
    const int ntop = (int)max(0LL, rt - rb);
    for (int idx = threadIdx.x; idx < n * ntop; idx += NT) {
      const int c = idx / ntop;
      const long long r = rb + (idx - c * ntop);
      W[(long long)c * rows + r] = WA(c, r);
    }
  }
  pc.lap(P.ctl, 9);
  // Compact WY form Q = I - Vh T Vh^H, built from the unit-norm reflectors vh_j = v_j / |v_j|
  // (tau = 2): a column just above the null threshold has |v_j| ~ 1e-8 |M| and tau_j ~ 1e16,
  // and the unnormalised form would chain such factors through T and lose orthogonality.
  // Gram of the unit reflectors: G[a][b] = vh_a^H vh_b over rows r >= max(a, b), a <= b;
  // per pair a walk over the own rows with two accumulator sets
  {
    const int n2 = n * n;
    double* mine = red[rp];
    rp ^= 1;
    for (int pidx = threadIdx.x; pidx < n2; pidx += NT) {
      const int a = pidx / n, b = pidx - (pidx / n) * n;
      double g0r = 0, g0i = 0, g1r = 0, g1i = 0;
      if (a <= b && qs.tau[a] != 0.0 && qs.tau[b] != 0.0) {
        long long r = max(rb, (long long)b);
        for (; r + 1 < re; r += 2) {
          const double2 va0 = (r == a) ? qs.vhead[a] : WA(a, r);
          const double2 vb0 = (r == b) ? qs.vhead[b] : WA(b, r);
          const double2 va1 = WA(a, r + 1);
          const double2 vb1 = (r + 1 == b) ? qs.vhead[b] : WA(b, r + 1);
          g0r = fma(va0.x, vb0.x, fma(va0.y, vb0.y, g0r));
          g0i = fma(va0.x, vb0.y, fma(-va0.y, vb0.x, g0i));
          g1r = fma(va1.x, vb1.x, fma(va1.y, vb1.y, g1r));
          g1i = fma(va1.x, vb1.y, fma(-va1.y, vb1.x, g1i));
        }
        if (r < re) {
          const double2 va0 = (r == a) ? qs.vhead[a] : WA(a, r);
          const double2 vb0 = (r == b) ? qs.vhead[b] : WA(b, r);
          g0r = fma(va0.x, vb0.x, fma(va0.y, vb0.y, g0r));
          g0i = fma(va0.x, vb0.y, fma(-va0.y, vb0.x, g0i));
        }
      }
      mine[2 * pidx] = g0r + g1r;
      mine[2 * pidx + 1] = g0i + g1i;
    }
    team_reduce_vec(tm, mine, redo, 2 * n2);
    for (int pidx = threadIdx.x; pidx < n2; pidx += NT) {
      const int a = pidx / n, b = pidx - (pidx / n) * n;
      if (a > b) continue;
      const double sab = qs.shat[a] * qs.shat[b];
      const double gr = sab * redo[2 * pidx], gi = sab * redo[2 * pidx + 1];
      G[a * ldg + b] = make_double2(gr, gi);
      G[b * ldg + a] = make_double2(gr, -gi);
    }
    __syncthreads();
  }
  pc.lap(P.ctl, 10);
  // T (upper triangular): T[j][j] = 2, T[0:j, j] = -2 T[0:j, 0:j] G[0:j, j] (rows and columns
  // of identity reflectors stay zero)
  for (int idx = threadIdx.x; idx < n * n; idx += NT) Tm[idx / n * ldg + idx % n] = make_double2(0, 0);
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const double tj = qs.tau[j] != 0.0 ? 2.0 : 0.0;
    if (threadIdx.x < j && tj != 0.0) {
      const int i = threadIdx.x;
      double sr0 = 0, si0 = 0, sr1 = 0, si1 = 0;  // two chains (FP64 latency)
      int k = i;
      for (; k + 1 < j; k += 2) {
        const double2 t0 = Tm[i * ldg + k], g0 = G[k * ldg + j];
        const double2 t1 = Tm[i * ldg + k + 1], g1 = G[(k + 1) * ldg + j];
        sr0 = fma(t0.x, g0.x, fma(-t0.y, g0.y, sr0));
        si0 = fma(t0.x, g0.y, fma(t0.y, g0.x, si0));
        sr1 = fma(t1.x, g1.x, fma(-t1.y, g1.y, sr1));
        si1 = fma(t1.x, g1.y, fma(t1.y, g1.x, si1));
      }
      if (k < j) {
        const double2 t0 = Tm[i * ldg + k], g0 = G[k * ldg + j];
        sr0 = fma(t0.x, g0.x, fma(-t0.y, g0.y, sr0));
        si0 = fma(t0.x, g0.y, fma(t0.y, g0.x, si0));
      }
      Tm[i * ldg + j] = make_double2(-tj * (sr0 + sr1), -tj * (si0 + si1));
    }
    if (threadIdx.x == 0) Tm[j * ldg + j] = make_double2(tj, 0.0);
    __syncthreads();
  }
  // Z[j][c] = shat_j sum_{j <= i <= c} T[j][i] shat_i conj(V[c][i]), so that
  // Q = I - V Z with the unnormalised V stored in the workspace
  for (int idx = threadIdx.x; idx < n * n; idx += NT) {
    const int j = idx / n, c = idx % n;
    double zr = 0, zi = 0;
    for (int i = j; i <= c; ++i) {
      if (qs.tau[i] == 0.0) continue;
      const double2 t = Tm[j * ldg + i];
      const double2 v = (c == i) ? qs.vhead[i] : W[(long long)i * rows + c];
      const double si = qs.shat[i];
      const double2 vci = make_double2(si * v.x, si * v.y);
      zr += t.x * vci.x + t.y * vci.y;
      zi += t.y * vci.x - t.x * vci.y;
    }
    Z[j * ldg + c] = make_double2(qs.shat[j] * zr, qs.shat[j] * zi);
  }
  pc.lap(P.ctl, 11);
  // phases of the diagonal of R
  for (int j = threadIdx.x; j < n; j += NT) {
    const double2 a = qs.rdiag[j];
    const double aa = sqrt(a.x * a.x + a.y * a.y);
    qs.ph[j] = aa > 0.0 ? make_double2(a.x / aa, a.y / aa) : make_double2(1.0, 0.0);
  }
  __syncthreads();
  // R (row j scaled by conj(ph_j)) into the bond buffer: R[j][k] = W[k][j] (k > j), diag alpha_j,
  // rescaled to ||R||_F = ||M||_F (the weight of dropped sub-columns returns to the kept content)
  if (tm.rank == 0) {
    __shared__ double s_rn[NWARP];
    double loc = 0.0;
    for (int idx = threadIdx.x; idx < n * n; idx += NT) {
      const int j = idx / n, k = idx % n;
      double2 r = make_double2(0, 0);
      if (k > j) r = W[(long long)k * rows + j];
      else if (k == j) r = qs.rdiag[j];
      loc = fma(r.x, r.x, fma(r.y, r.y, loc));
    }
    loc = warp_sum(loc);
    if (lane == 0) s_rn[warp] = loc;
    __syncthreads();
    double rn = 0.0;
    for (int w = 0; w < NWARP; ++w) rn += s_rn[w];
    const double scale = rn > 0.0 ? fro_m / sqrt(rn) : 1.0;
    for (int idx = threadIdx.x; idx < n * n; idx += NT) {
      const int j = idx / n, k = idx % n;
      double2 r = make_double2(0, 0);
      if (k > j) r = W[(long long)k * rows + j];
      else if (k == j) r = qs.rdiag[j];
      const double2 p = qs.ph[j];
      Rout[idx] = make_double2(scale * (r.x * p.x + r.y * p.y), scale * (r.y * p.x - r.x * p.y));
    }
  }
  // Q[r][c] = (delta_rc - sum_j V[r][j] Z[j][c]) * ph_c over the own rows, one (c, r) pair
  // per thread, written back into the tensor; V[r][j] = 0 for j > r and Z[j][c] = 0 for
  // j > c, so j runs to min(r, c)
  for (int idx = threadIdx.x; idx < n * nr; idx += NT) {
    const int c = fdivu(idx, nr, inv_nr);
    const long long r = rb + (idx - c * nr);
    const int jmax = (int)(r < (long long)c ? r : (long long)c);
    double qre = (r == c) ? 1.0 : 0.0, qim = 0.0;
    for (int j = 0; j <= jmax; ++j) {
      if (qs.tau[j] == 0.0) continue;
      const double2 vr = (r == j) ? qs.vhead[j] : WA(j, r);
      const double2 z = Z[j * ldg + c];
      qre -= vr.x * z.x - vr.y * z.y;
      qim -= vr.x * z.y + vr.y * z.x;
    }
    const double2 p = qs.ph[c];
    A[qr_addr(nd, l, r, c)] = make_double2(qre * p.x - qim * p.y, qre * p.y + qim * p.x);
  }
  team_sync(tm);
  pc.lap(P.ctl, 12);
}

#include "qr_ds.cuh"

// ------------------------------------------------------------------ absorb
// A_u <- R applied on leg I.leg (FP64), through a temporary
__device__ __noinline__ void op_absorb(const KernelParams& P, Team& tm, const Instr& I, double2* work) {
  const NodeDesc nd = P.nodes[I.node];
  const long long N = nd.size;
  double2* A = P.pool + nd.off;
  const double2* R = P.pool + P.trees[I.tree].bond_off;
  const int l = I.leg;
  for (long long idx = tm.gtid(); idx < N; idx += tm.nthr()) {
    LegPos lp = leg_pos(nd, l, idx);
    auto a = mode_dot<double>(R + (long long)lp.i * nd.dims[l], nd.dims[l], A, lp.base, nd.strides[l]);
    work[idx] = a;
  }
  team_sync(tm);
  for (long long idx = tm.gtid(); idx < N; idx += tm.nthr()) A[idx] = work[idx];
  team_sync(tm);
}

// ------------------------------------------------------------------ environment update
// env(u -> v): block 0 = Q^H (H-terms of u without v) Q, block 1+b = Q^H (channel factor b) Q,
// contracted over every leg of Q except the leg toward v.
template <typename T>
__device__ __noinline__ void op_env(const KernelParams& P, Team& tm, const Instr& I, double2* work) {
  const NodeDesc nd = P.nodes[I.node];
  const TermList L = P.lists[I.terms];
  const long long N = nd.size;
  const long long kv = P.kvec;
  using V = typename C2<T>::t;
  const double2* Q = P.pool + nd.off;
  auto* tmp = reinterpret_cast<V*>(work + (long long)P.mmax * kv);
  V* Y = reinterpret_cast<V*>(work);  // Y_0 .. Y_nchan at Y + b*kv, compute type (fits: 1 + nchan <= mmax)
  PhaseClock pc;
  pc.start(P.profile && tm.rank == 0 && threadIdx.x == 0, tm.kind == TEAM_GRID);
  const int l = I.leg;
  const int D = I.D;
  const int nb = 1 + I.nchan;
  OpStage& os = s_os;
  stage_op<T>(P, I, L, P.chans + I.chan_first, I.nchan, os);
  V* xs = vec_smem<T>(P, os, N);
  // the operand Q in the compute type: shared memory when it fits, else (mixed precision) a
  // converted copy in the workspace, else (FP64) the tensor itself
  const V* xq;
  if (xs) {
    stage_vector<T>(xs, Q, N);
    xq = xs;
  } else if constexpr (!std::is_same<T, double>::value) {
    V* qf = reinterpret_cast<V*>(work + (long long)(P.mmax + P.n_tmp) * kv);
    for (long long idx = tm.gtid(); idx < N; idx += tm.nthr()) qf[idx] = cvt<T>(Q[idx]);
    team_sync(tm);
    xq = qf;
  } else {
    xq = reinterpret_cast<const V*>(Q);
  }
  pc.lap(P.ctl, 16);
  if (L.n2 > 0) {
    apply_stage1<T>(P, tm, nd, xq, L, tmp, kv, os);
    team_sync(tm);
  }
  for (long long idx = tm.gtid(); idx < N; idx += tm.nthr()) {
    Y[idx] = apply_stage2_at<T>(P, nd, xq, L, tmp, kv, idx, os);
    for (int b = 0; b < I.nchan; ++b) Y[(long long)(1 + b) * kv + idx] = factor_dot<T>(P, nd, os.chans[b], os, xq, idx);
  }
  team_sync(tm);
  pc.lap(P.ctl, 17);
  // projection: out[b][a][a'] = sum_rows conj(Q[row, a]) Y_b[row, a'].  Each CTA owns a
  // contiguous block of the output values and sums them over all rows: the rows of an output
  // are split into `parts` ranges over the CTA's threads (partial sums in the compute type in
  // runs of 64 rows, then FP64), and one thread per output adds its parts in a fixed order and
  // writes the value; no partial sums cross CTAs.
  const long long rows = N / D;
  const int nval = nb * D * D;
  const long long lst = nd.strides[l];
  const int opc = (nval + tm.size - 1) / tm.size;
  const int ob = min(nval, tm.rank * opc), oe = min(nval, ob + opc);
  const int nout = oe - ob;
  const int parts = nout > 0 ? max(1, min(16, NT / nout)) : 1;
  const long long rpp = (rows + parts - 1) / parts;
  double2* pbuf = P.cta_scratch + (long long)blockIdx.x * P.cta_scratch_stride;  // parts x nout (parts > 1)
  double2* out = P.pool + I.env_out;
  for (int it = threadIdx.x; it < nout * parts; it += NT) {
    const int o = ob + it % nout, part = it / nout;
    const int b = o / (D * D);
    const int a = (o / D) % D;
    const int a2 = o % D;
    const V* Yb = Y + (long long)b * kv;
    const long long rb0 = part * rpp, re0 = min(rows, rb0 + rpp);
    double accr = 0, acci = 0;
    for (long long r0 = rb0; r0 < re0; r0 += 64) {
      V s0, s1;
      s0.x = s0.y = s1.x = s1.y = 0;
      const long long r1 = min(re0, r0 + 64);
      long long r = r0;
      for (; r + 1 < r1; r += 2) {  // two rows at a time: independent accumulators
        const long long p0 = fdivu((int)r, (int)lst, nd.inv_strides[l]), q0 = r - p0 * lst;
        const long long p1 = fdivu((int)(r + 1), (int)lst, nd.inv_strides[l]), q1 = r + 1 - p1 * lst;
        const long long base0 = p0 * D * lst + q0, base1 = p1 * D * lst + q1;
        const V qa0 = xq[base0 + (long long)a * lst], y0 = Yb[base0 + (long long)a2 * lst];
        const V qa1 = xq[base1 + (long long)a * lst], y1 = Yb[base1 + (long long)a2 * lst];
        s0.x = fma(qa0.x, y0.x, fma(qa0.y, y0.y, s0.x));
        s0.y = fma(qa0.x, y0.y, fma(-qa0.y, y0.x, s0.y));
        s1.x = fma(qa1.x, y1.x, fma(qa1.y, y1.y, s1.x));
        s1.y = fma(qa1.x, y1.y, fma(-qa1.y, y1.x, s1.y));
      }
      if (r < r1) {
        const long long p0 = fdivu((int)r, (int)lst, nd.inv_strides[l]), q0 = r - p0 * lst;
        const long long base0 = p0 * D * lst + q0;
        const V qa0 = xq[base0 + (long long)a * lst], y0 = Yb[base0 + (long long)a2 * lst];
        s0.x = fma(qa0.x, y0.x, fma(qa0.y, y0.y, s0.x));
        s0.y = fma(qa0.x, y0.y, fma(-qa0.y, y0.x, s0.y));
      }
      accr += (double)s0.x + (double)s1.x;
      acci += (double)s0.y + (double)s1.y;
    }
    if (parts == 1) {
      out[o] = make_double2(accr, acci);
      if constexpr (!std::is_same<T, double>::value) P.pool32[I.env_out + o] = make_float2((float)accr, (float)acci);
    } else
      pbuf[(long long)part * nout + (o - ob)] = make_double2(accr, acci);  // parts * nout <= NT
  }
  __syncthreads();
  pc.lap(P.ctl, 18);
  if (parts > 1)
    for (int k = threadIdx.x; k < nout; k += NT) {
      double sr = 0.0, si = 0.0;
      for (int part = 0; part < parts; ++part) {
        const double2 v = pbuf[(long long)part * nout + k];
        sr += v.x;
        si += v.y;
      }
      out[ob + k] = make_double2(sr, si);
      if constexpr (!std::is_same<T, double>::value) P.pool32[I.env_out + ob + k] = make_float2((float)sr, (float)si);
    }
  team_sync(tm);
  pc.lap(P.ctl, 19);
  if (tm.rank == 0 && threadIdx.x == 0) {
    atomicAdd(&P.ctl->applies, 1ull);
    atomicAdd(&P.ctl->flops, I.flops);
  }
}

// ------------------------------------------------------------------ record rho_S
__device__ __noinline__ void op_record(const KernelParams& P, Team& tm, const Instr& I, int* counter) {
  const TreeDesc td = P.trees[I.tree];
  if (td.traj_off < 0) return;
  const NodeDesc nd = P.nodes[td.node0];
  const int ne = td.n_el;
  const long long rows = nd.size / ne;  // phys leg is the last leg: stride 1
  const double2* A = P.pool + nd.off;
  const int nval = ne * ne;
  double* part = team_partials(tm);
  const long long chunk = (rows + tm.size - 1) / tm.size;
  const long long r_begin = (long long)tm.rank * chunk, r_end = min(rows, r_begin + chunk);
  for (int o = threadIdx.x; o < nval; o += NT) {
    const int s1 = o / ne, s2 = o % ne;
    double accr = 0, acci = 0;
    for (long long r = r_begin; r < r_end; ++r) {
      double2 a = A[r * ne + s1], b = A[r * ne + s2];
      accr = fma(a.x, b.x, fma(a.y, b.y, accr));
      acci = fma(a.y, b.x, fma(-a.x, b.y, acci));
    }
    part[(long long)tm.rank * 2 * nval + 2 * o] = accr;
    part[(long long)tm.rank * 2 * nval + 2 * o + 1] = acci;
  }
  int slot = *counter;
  if (slot >= P.max_record) slot = P.max_record - 1;
  team_finish_multi(tm, 2 * nval, (double*)(P.pool + td.traj_off + (long long)slot * nval), 1.0);
  if (tm.rank == 0 && threadIdx.x == 0) {
    *counter = *counter + 1;
    atomicAdd(&P.ctl->steps, 1ull);
  }
}

// ------------------------------------------------------------------ interpreter
template <typename T>
__device__ void exec_op(const KernelParams& P, Team& tm, const Instr& I, double2* work);

template <typename T>
__device__ void exec(const KernelParams& P, Team& tm, const Instr& I, double2* work) {
  if (!P.profile) {
    exec_op<T>(P, tm, I, work);
    return;
  }
  const long long t0 = clock64();
  exec_op<T>(P, tm, I, work);
  if (tm.rank == 0 && threadIdx.x == 0) {
    const long long dt = clock64() - t0;
    atomicAdd(&P.ctl->prof_cycles[I.op][tm.kind], (unsigned long long)dt);
    atomicAdd(&P.ctl->prof_count[I.op][tm.kind], 1ull);
  }
}

template <typename T>
__device__ void exec_op(const KernelParams& P, Team& tm, const Instr& I, double2* work) {
  const double tau = 0.5 * P.dt;
  switch (I.op) {
    case OP_FWD:
    case OP_BOND:
      if (!(tm.kind == TEAM_CLUSTER && P.cluster_resident && op_expm_cluster<T>(P, tm, I, tau)))
        op_expm<T>(P, tm, I, work, tau);
      break;
    case OP_QR:
      if (P.precision != 0)
        op_qr_ds(P, tm, I, work);
      else
        op_qr(P, tm, I, work);
      break;
    case OP_ENV:
      op_env<T>(P, tm, I, work);
      break;
    case OP_ABSORB:
      if (P.precision != 0)
        op_absorb_ds(P, tm, I, work);
      else
        op_absorb(P, tm, I, work);
      break;
    case OP_RECORD:
      op_record(P, tm, I, P.traj_count + I.tree);
      break;
  }
}

template <typename T>
__device__ void run(const KernelParams& P, int phase) {
  const int cs = P.cluster_ctas;
  const int cluster_id = blockIdx.x / cs;
  const int n_clusters = gridDim.x / cs;
  const int crank = (int)cg::this_cluster().block_rank();
  Team ct;
  ct.kind = TEAM_CLUSTER;
  ct.rank = crank;
  ct.size = cs;
  ct.red = P.red + (long long)cluster_id * 2 * P.red_stride;
  ct.red_stride = P.red_stride;
  ct.parity = 0;
  ct.ctl = P.ctl;
  ct.spin_limit = P.spin_limit;
  ct.csize = cs;
  double2* cwork = P.work + (long long)cluster_id * P.work_stride;
  if (P.batched) {
    for (int tree = cluster_id; tree < P.n_trees; tree += n_clusters) {
      const TreeDesc& td = P.trees[tree];
      const int first = phase == 0 ? td.init_first : (phase == 2 ? td.obs_first : (phase == 3 ? td.grow_first : td.prog_first));
      const int count = phase == 0 ? td.init_count : (phase == 2 ? td.obs_count : (phase == 3 ? td.grow_count : td.prog_count));
      const int nst = phase == 1 ? P.n_steps : 1;
      for (int s = 0; s < nst; ++s) {
        for (int k = 0; k < count; ++k) {
          exec<T>(P, ct, P.prog[first + k], cwork);
        }
      }
    }
    return;
  }
  Team gt;
  gt.kind = TEAM_GRID;
  gt.rank = blockIdx.x;
  gt.size = gridDim.x;
  gt.red = P.red_grid;
  gt.red_stride = P.red_stride_grid;
  gt.parity = 0;
  gt.ctl = P.ctl;
  gt.spin_limit = P.spin_limit;
  gt.csize = cs;
  const TreeDesc& td = P.trees[0];
  const int first = phase == 0 ? td.init_first : (phase == 2 ? td.obs_first : (phase == 3 ? td.grow_first : td.prog_first));
  const int count = phase == 0 ? td.init_count : (phase == 2 ? td.obs_count : (phase == 3 ? td.grow_count : td.prog_count));
  const int nst = phase == 1 ? P.n_steps : 1;
  int prev = TEAM_GRID;
  for (int s = 0; s < nst; ++s) {
    for (int k = 0; k < count; ++k) {
      const Instr& I = P.prog[first + k];
      if (I.team == TEAM_GRID) {
        if (prev == TEAM_CLUSTER) grid_sync(P.ctl, P.spin_limit);
        exec<T>(P, gt, I, P.work);
      } else if (cluster_id == 0) {
        exec<T>(P, ct, I, cwork);
        if (crank == 0 && threadIdx.x == 0) atomicAdd(&P.ctl->progress, 1u);
      }
      prev = I.team;
    }
  }
  if (prev == TEAM_CLUSTER) grid_sync(P.ctl, P.spin_limit);
}

__device__ __forceinline__ unsigned sreg_cluster_nctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned sreg_dynamic_smem_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
  return r;
}

__global__ void __launch_bounds__(NT, 1) k_sweep(KernelParams P, int phase) {
  // Launch self-check before any barrier or distributed-shared-memory access: the
  // interpreter addresses cluster peers by rank and stages operands up to smem_bytes, so a
  // launch with another cluster shape or less dynamic shared memory returns an error
  // status instead of running.  Every CTA takes the same decision.
  const unsigned ncta = sreg_cluster_nctarank();
  if (ncta != (unsigned)P.cluster_ctas || (long long)sreg_dynamic_smem_size() < P.smem_bytes ||
      gridDim.x % (unsigned)P.cluster_ctas != 0) {
    if (threadIdx.x == 0 && blockIdx.x == 0) set_status(P.ctl, ST_LAUNCH, 300, (int)ncta);
    return;
  }
  // tensor memory for the split-precision contractions (one 128-column accumulator per CTA)
  const bool tc_on = P.precision == 1 || P.precision == 2;
  if (threadIdx.x == 0) s_tc.on = 0;
  if (tc_on) {
    if ((threadIdx.x >> 5) == 0) tc::tmem_alloc(&s_tc.tmem, kTcTmemCols);
    if (threadIdx.x == 0) {
      tc::mbar_init(&s_tc.mbar, 1);
      s_tc.phase = 0;
      s_tc.on = 1;
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
  }
  __syncthreads();
  if (P.precision == 0)
    run<double>(P, phase);
  else
    run<float>(P, phase);
  if (tc_on) {
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(s_tc.tmem, kTcTmemCols);
  }
}

// ------------------------------------------------------------------ observables
// Bond or site density of node v's leg l from the incoming parent-bond density rho_in
// (D_p x D_p, or nullptr at the root):
//   out[b][b'] = sum rho_in[p', p] A[p, .., b, ..] conj(A[p', .., b', ..]) over the other legs.
// One CTA per call (small sizes), except that the root (rho_in == nullptr) may be large:
// a grid of CTAs writes partials, reduced by k_reduce_partials.
// X = rho_in applied on leg 0 of the node tensor: X[idx] = sum_a' rho_in[a'][a] A[.., a', ..]
// with a the leg-0 index of idx (the incoming parent-bond density of a downward pass)
__global__ void k_apply_rho0(const double2* A, NodeDesc nd, const double2* rho_in, double2* X) {
  const int Dp = nd.dims[0];
  const long long stp = nd.strides[0];
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nd.size;
       idx += (long long)gridDim.x * blockDim.x) {
    const int qa = fdivu((int)idx, (int)stp, nd.inv_strides[0]);
    const int a = qa - fdivu(qa, Dp, nd.inv_dims[0]) * Dp;
    const long long b0 = idx - (long long)a * stp;
    double xr = 0.0, xi = 0.0;
    for (int a2 = 0; a2 < Dp; ++a2) {
      const double2 r_ = rho_in[a2 * Dp + a];
      const double2 v = A[b0 + (long long)a2 * stp];
      xr = fma(r_.x, v.x, fma(-r_.y, v.y, xr));
      xi = fma(r_.x, v.y, fma(r_.y, v.x, xi));
    }
    X[idx] = make_double2(xr, xi);
  }
}

// partials of rho[b][b2] = sum_rows X[row, b] conj(A[row, b2]) along leg l, rows split over
// the blocks (X = A for the root)
__global__ void k_density_partial(const double2* X, const double2* A, NodeDesc nd, int l, double* partials) {
  const int D = nd.dims[l];
  const long long N = nd.size;
  const long long st = nd.strides[l];
  const long long rows = N / D;
  const long long chunk = (rows + gridDim.x - 1) / gridDim.x;
  const long long r_begin = (long long)blockIdx.x * chunk, r_end = min(rows, r_begin + chunk);
  for (int o = threadIdx.x; o < D * D; o += blockDim.x) {
    const int b = o / D, b2 = o % D;
    double accr = 0, acci = 0;
    for (long long r = r_begin; r < r_end; ++r) {
      const long long p = fdivu((int)r, (int)st, nd.inv_strides[l]), q = r - p * st;
      const long long base = p * D * st + q;
      const double2 y = A[base + (long long)b2 * st];
      const double2 xa = X[base + (long long)b * st];
      accr = fma(xa.x, y.x, fma(xa.y, y.y, accr));
      acci = fma(xa.y, y.x, fma(-xa.x, y.y, acci));
    }
    partials[(long long)blockIdx.x * 2 * D * D + 2 * o] = accr;
    partials[(long long)blockIdx.x * 2 * D * D + 2 * o + 1] = acci;
  }
}

__global__ void k_reduce_partials(const double* partials, int nblocks, int nval, double* out) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nval; k += gridDim.x * blockDim.x) {
    double s = 0;
    for (int b = 0; b < nblocks; ++b) s += partials[(long long)b * nval + k];
    out[k] = s;
  }
}

// <n> = sum_s s Re(rho[s][s]) of one site density
__global__ void k_occ(const double2* dens, int d, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double o = 0;
    for (int q = 1; q < d; ++q) o += q * dens[q * d + q].x;
    *out = o;
  }
}

// norm^2 and <A|H_eff|A> at the root with FP64 terms
__global__ void k_energy_partial(KernelParams P, int node, int terms, double* partials) {
  const NodeDesc nd = P.nodes[node];
  const TermList L = P.lists[terms];
  const double2* x = P.pool + nd.off;
  const long long N = nd.size;
  double e = 0, nn = 0;
  OpStage& os = s_os;
  const int nt = L.count < TTNS_MAX_TERMS ? L.count : TTNS_MAX_TERMS;
  for (int t = threadIdx.x; t < nt; t += blockDim.x) os.terms[t] = P.terms[L.first + t];
  if (threadIdx.x == 0) {
    os.a_off = os.b_off = 0;
    os.a_n = os.b_n = 0;
    os.end = 0;
  }
  __syncthreads();
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += (long long)gridDim.x * blockDim.x) {
    auto a = apply_stage2_at<double>(P, nd, x, L, P.work + (long long)P.mmax * P.kvec, P.kvec, idx, os);
    double2 v = x[idx];
    e = fma(v.x, a.x, fma(v.y, a.y, e));
    nn = fma(v.x, v.x, fma(v.y, v.y, nn));
  }
  __shared__ double s1[NWARP], s2[NWARP];
  e = warp_sum(e);
  nn = warp_sum(nn);
  if ((threadIdx.x & 31) == 0) { s1[threadIdx.x >> 5] = e; s2[threadIdx.x >> 5] = nn; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int w = 0; w < NWARP; ++w) { a += s1[w]; b += s2[w]; }
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
  }
}

// stage 1 of a term list over a whole tensor, written to the worker-0 temporaries
__global__ void k_stage1(KernelParams P, int node, int terms) {
  const NodeDesc nd = P.nodes[node];
  const TermList L = P.lists[terms];
  const Term* tl = P.terms + L.first + (L.count - L.n2);
  const double2* x = P.pool + nd.off;
  double2* tmp = P.work + (long long)P.mmax * P.kvec;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nd.size; idx += (long long)gridDim.x * blockDim.x) {
    for (int t = 0; t < L.n2; ++t) {
      const Factor f = tl[t].f[0];
      LegPos lp = leg_pos(nd, f.leg, idx);
      auto a = mode_dot<double>(P.pool + f.mat + (long long)lp.i * nd.dims[f.leg], nd.dims[f.leg], x, lp.base,
                                nd.strides[f.leg]);
      tmp[t * P.kvec + idx] = a;
    }
  }
}

// H x for an explicit input x with a node's term list (FP64): stage 1 of the two-stage terms
// into the worker-0 temporaries, then y = the sum of all terms
__global__ void k_stage1_x(KernelParams P, int node, int terms, const double2* x) {
  const NodeDesc nd = P.nodes[node];
  const TermList L = P.lists[terms];
  const Term* tl = P.terms + L.first + (L.count - L.n2);
  double2* tmp = P.work + (long long)P.mmax * P.kvec;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nd.size;
       idx += (long long)gridDim.x * blockDim.x) {
    for (int t = 0; t < L.n2; ++t) {
      const Factor f = tl[t].f[0];
      LegPos lp = leg_pos(nd, f.leg, idx);
      tmp[t * P.kvec + idx] = mode_dot<double>(P.pool + f.mat + (long long)lp.i * nd.dims[f.leg], nd.dims[f.leg], x,
                                               lp.base, nd.strides[f.leg]);
    }
  }
}

__global__ void k_apply_x(KernelParams P, int node, int terms, const double2* x, double2* y) {
  const NodeDesc nd = P.nodes[node];
  const TermList L = P.lists[terms];
  OpStage& os = s_os;
  const int nt = L.count < TTNS_MAX_TERMS ? L.count : TTNS_MAX_TERMS;
  for (int t = threadIdx.x; t < nt; t += blockDim.x) os.terms[t] = P.terms[L.first + t];
  if (threadIdx.x == 0) {
    os.a_off = os.b_off = 0;
    os.a_n = os.b_n = 0;
    os.end = 0;
  }
  __syncthreads();
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nd.size;
       idx += (long long)gridDim.x * blockDim.x)
    y[idx] = apply_stage2_at<double>(P, nd, x, L, P.work + (long long)P.mmax * P.kvec, P.kvec, idx, os);
}

cudaError_t launch_apply_x(const KernelParams& P, int node, int terms, int n2, const double2* x, double2* y,
                           int nblocks, cudaStream_t st) {
  if (n2 > 0) k_stage1_x<<<nblocks, NT, 0, st>>>(P, node, terms, x);
  k_apply_x<<<nblocks, NT, 0, st>>>(P, node, terms, x, y);
  return cudaGetLastError();
}

// Self-test of the bounded wait: two CTAs; with `skip` set the second CTA never
// arrives at the barrier, so the first one must give up after spin_limit cycles.
__global__ void k_wait_selftest(Ctl* ctl, long long spin_limit, int skip) {
  if (skip && blockIdx.x == 1) return;
  grid_sync(ctl, spin_limit);
}

cudaError_t launch_wait_selftest(Ctl* ctl, long long spin_limit, int skip, cudaStream_t st) {
  void* args[] = {&ctl, &spin_limit, &skip};
  return cudaLaunchCooperativeKernel((void*)k_wait_selftest, dim3(2), dim3(NT), args, 0, st);
}

// Copy of a node tensor into a tensor of the same legs with larger (or equal) dimensions,
// zero on the new indices (row-major, legs in the node's order)
__global__ void k_pad_copy(const double2* src, NodeDesc so, double2* dst, NodeDesc dn) {
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < dn.size;
       idx += (long long)gridDim.x * blockDim.x) {
    long long rem = idx, off = 0;
    bool in = true;
    for (int l = 0; l < dn.nl; ++l) {
      const long long i = rem / dn.strides[l];
      rem -= i * dn.strides[l];
      in = in && i < so.dims[l];
      off += i * so.strides[l];
    }
    dst[idx] = in ? src[off] : make_double2(0.0, 0.0);
  }
}

cudaError_t launch_pad_copy(const double2* src_pool, const NodeDesc& so, double2* dst_pool, const NodeDesc& dn,
                            cudaStream_t st) {
  long long nb = (dn.size + 255) / 256;
  nb = nb > 4096 ? 4096 : (nb < 1 ? 1 : nb);
  k_pad_copy<<<(int)nb, 256, 0, st>>>(src_pool + so.off, so, dst_pool + dn.off, dn);
  return cudaGetLastError();
}

// FP32 mirror of the pool (after the pool was written from the host)
__global__ void k_mirror32(const double2* pool, float2* pool32, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    pool32[i] = make_float2((float)pool[i].x, (float)pool[i].y);
}

cudaError_t launch_mirror32(const double2* pool, float2* pool32, long long n, cudaStream_t st) {
  long long nb = (n + 255) / 256;
  nb = nb > 4096 ? 4096 : (nb < 1 ? 1 : nb);
  k_mirror32<<<(int)nb, 256, 0, st>>>(pool, pool32, n);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ host launch helpers
static bool g_tables_set = false;

cudaError_t upload_constants() {
  if (g_tables_set) return cudaSuccess;
  double inv[256], invf[128];
  inv[0] = 0.0;
  for (int k = 1; k < 256; ++k) inv[k] = 1.0 / k;
  invf[0] = 1.0;
  for (int k = 1; k < 128; ++k) invf[k] = invf[k - 1] / k;
  cudaError_t e = cudaMemcpyToSymbol(c_inv, inv, sizeof(inv));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(c_invfact, invf, sizeof(invf));
  if (e == cudaSuccess) g_tables_set = true;
  return e;
}

cudaError_t launch_sweep(const KernelParams& P, int phase, int grid, int cluster, int cooperative,
                         cudaStream_t stream) {
  cudaError_t e = upload_constants();
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_sweep, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.smem_bytes);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = (size_t)P.smem_bytes;
  cfg.stream = stream;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeCooperative;
  at[1].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = cooperative ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, k_sweep, P, phase);
}

cudaError_t max_grid_for(int cluster, long long smem_bytes, int* grid) {
  cudaError_t e = cudaFuncSetAttribute(k_sweep, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = (size_t)smem_bytes;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int nclusters = 0;
  e = cudaOccupancyMaxActiveClusters(&nclusters, k_sweep, &cfg);
  if (e != cudaSuccess) return e;
  *grid = nclusters * cluster;
  return cudaSuccess;
}

cudaError_t launch_density(const double2* pool, const NodeDesc& nd, int l, const double2* rho_in, double2* xbuf,
                           double* partials, int nblocks, double* out, cudaStream_t st) {
  const double2* A = pool + nd.off;
  const double2* X = A;
  if (rho_in) {
    long long nb = (nd.size + NT - 1) / NT;
    nb = nb > 4096 ? 4096 : nb;
    k_apply_rho0<<<(int)nb, NT, 0, st>>>(A, nd, rho_in, xbuf);
    X = xbuf;
  }
  k_density_partial<<<nblocks, NT, 0, st>>>(X, A, nd, l, partials);
  const int D = nd.dims[l];
  k_reduce_partials<<<(2 * D * D + NT - 1) / NT, NT, 0, st>>>(partials, nblocks, 2 * D * D, out);
  return cudaGetLastError();
}

cudaError_t launch_occ(const double2* dens, int d, double* out, cudaStream_t st) {
  k_occ<<<1, 32, 0, st>>>(dens, d, out);
  return cudaGetLastError();
}

cudaError_t launch_energy(const KernelParams& P, int node, int terms, int n2, double* partials, int nblocks,
                          double* out, cudaStream_t st) {
  if (n2 > 0) k_stage1<<<nblocks, NT, 0, st>>>(P, node, terms);
  k_energy_partial<<<nblocks, NT, 0, st>>>(P, node, terms, partials);
  k_reduce_partials<<<1, NT, 0, st>>>(partials, nblocks, 2, out);
  return cudaGetLastError();
}

}  // namespace ttns
