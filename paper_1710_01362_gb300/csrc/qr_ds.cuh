// Householder QR of the mixed-precision modes in double-single arithmetic.
//
// Included by sweep.cu after op_qr: the same algorithm, completion rule and cutoff (null
// sub-columns get the identity reflector, R_jj = 0; compact WY form of Q from unit
// reflectors; R_jj made real >= 0; R rescaled to ||R||_F = ||M||_F), with the O(rows n^2)
// arithmetic (column dots, trailing updates, Gram matrix of the reflectors, the formation of
// Q) and the team reductions carried as unevaluated sums h + l of two floats.  This part
// issues FP32 operations at about 80 times its FP64 rate; the representation has a 48-bit
// significand and FP32's exponent range, and the error-free transformations below keep every
// sum and product to about 2^-44 relative, far below the FP32-class error of the mixed
// modes' contractions.  The scalar reflector arithmetic (square roots, divisions, the
// triangular factor T) stays in FP64.
//
// Error-free transformations: TwoSum (Knuth: s + e = a + b exactly) and TwoProduct through
// the fused multiply-add (p + e = a b exactly); the _rn intrinsics keep the compiler from
// contracting or reassociating them.  Products accumulate as a running float sum plus a
// float sum of all rounding errors, renormalised once at the end (the compensated dot
// product of Ogita, Rump and Oishi, SIAM J. Sci. Comput. 26 (2005), with double-single
// inputs).
//
// A value below 2^-126 (about 1.2e-38) is zero here, so a Householder head below it counts as
// zero (phase 1), where the FP64 path draws that line at 1e-280.

// Conversions by integer arithmetic on the bit patterns (the FP64 <-> FP32 conversion
// instructions run on the narrow FP64 pipe).  ds_from: the head is the double rounded to
// nearest-even float (from the 29 dropped significand bits), the tail the exact remainder
// rounded to a float, scaled by a power of two; values below 2^-126 give zero, values beyond
// FP32's range take the conversion instruction.  Identical to h = (float) x,
// l = (float) (x - h) for |x| >= 2^-74.
__device__ __forceinline__ float magic_i2f(int n) {  // exact for |n| < 2^22
  return __uint_as_float(0x4B400000u + (unsigned)n) - 12582912.0f;
}
__device__ __forceinline__ float2 ds_from(double x) {
  const unsigned hi32 = (unsigned)__double2hiint(x), lo32 = (unsigned)__double2loint(x);
  const int e = (int)((hi32 >> 20) & 0x7FFu);
  if (e < 897) return make_float2(0.f, 0.f);
  if (e > 1149) return make_float2(__double2float_rn(x), 0.f);
  unsigned fb = (hi32 & 0x80000000u) | ((unsigned)(e - 896) << 23) | ((hi32 & 0xFFFFFu) << 3) | (lo32 >> 29);
  const unsigned rest = lo32 & 0x1FFFFFFFu;
  const unsigned up = (rest > 0x10000000u) || (rest == 0x10000000u && (fb & 1u));
  fb += up;  // a carry into the exponent field is the correct rounding
  const int lrem = (int)rest - (int)(up << 29);  // x - h in units of 2^(e - 1075)
  float l = __fmaf_rn(magic_i2f(lrem >> 14), 16384.0f, magic_i2f(lrem & 0x3FFF));
  const int se = e - 948;
  l = se >= 1 ? __fmul_rn(l, __uint_as_float((unsigned)se << 23))
              : __fmul_rn(__fmul_rn(l, 5.421010862427522e-20f), __uint_as_float((unsigned)(se + 64) << 23));
  if (hi32 & 0x80000000u) l = -l;
  return make_float2(__uint_as_float(fb), l);
}
// float -> double by the bit pattern (zero and normal floats; others by the instruction)
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ef = (u >> 23) & 0xFFu;
  if ((u << 1) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
  if (ef == 0u || ef == 255u) return (double)f;
  return __hiloint2double((int)((u & 0x80000000u) | ((ef + 896u) << 20) | ((u & 0x7FFFFFu) >> 3)), (int)((u & 7u) << 29));
}
__device__ __forceinline__ double ds_to(float2 a) { return f2d_bits(a.x) + f2d_bits(a.y); }
// s + t renormalised to a head and a tail (exact when |s| >= |t|)
__device__ __forceinline__ float2 ds_quick(float s, float t) {
  const float h = __fadd_rn(s, t);
  return make_float2(h, __fsub_rn(t, __fsub_rn(h, s)));
}
__device__ __forceinline__ float2 ds_add(float2 a, float2 b) {
  const float s = __fadd_rn(a.x, b.x);
  const float v = __fsub_rn(s, a.x);
  const float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, v)), __fsub_rn(b.x, v));
  return ds_quick(s, __fadd_rn(e, __fadd_rn(a.y, b.y)));
}
__device__ __forceinline__ float2 ds_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 ds_re(float4 z) { return make_float2(z.x, z.y); }
__device__ __forceinline__ float2 ds_im(float4 z) { return make_float2(z.z, z.w); }
__device__ __forceinline__ float4 ds_c(float2 re, float2 im) { return make_float4(re.x, re.y, im.x, im.y); }
__device__ __forceinline__ float4 ds_cfrom(double2 z) { return ds_c(ds_from(z.x), ds_from(z.y)); }
__device__ __forceinline__ double2 ds_cto(float4 z) { return make_double2(ds_to(ds_re(z)), ds_to(ds_im(z))); }

struct DsAcc {
  float s, c;  // running sum and the sum of its rounding errors
  __device__ __forceinline__ void init(float2 a) {
    s = a.x;
    c = a.y;
  }
  __device__ __forceinline__ void mac(float2 x, float2 y) {  // += x y (the lo*lo term is below the format)
    const float p = __fmul_rn(x.x, y.x);
    float e = __fmaf_rn(x.x, y.x, -p);
    e = __fmaf_rn(x.x, y.y, e);
    e = __fmaf_rn(x.y, y.x, e);
    const float t = __fadd_rn(s, p);
    const float v = __fsub_rn(t, s);
    c = __fadd_rn(c, __fadd_rn(__fadd_rn(__fsub_rn(s, __fsub_rn(t, v)), __fsub_rn(p, v)), e));
    s = t;
  }
  __device__ __forceinline__ float2 val() const { return ds_quick(s, c); }
};

// complex accumulators: (ar, ai) += conj(v) w, and (ar, ai) += a b
__device__ __forceinline__ void ds_conj_mac(DsAcc& ar, DsAcc& ai, float4 v, float4 w) {
  ar.mac(ds_re(v), ds_re(w));
  ar.mac(ds_im(v), ds_im(w));
  ai.mac(ds_re(v), ds_im(w));
  ai.mac(ds_neg(ds_im(v)), ds_re(w));
}
__device__ __forceinline__ void ds_cmac(DsAcc& ar, DsAcc& ai, float4 a, float4 b) {
  ar.mac(ds_re(a), ds_re(b));
  ar.mac(ds_neg(ds_im(a)), ds_im(b));
  ai.mac(ds_re(a), ds_im(b));
  ai.mac(ds_im(a), ds_re(b));
}

__device__ __forceinline__ float2 shfl_xor_ds(float2 v, int o) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}

// warp_reduce_t for double-single values: lane L returns the total of value
// warp_reduce_vid<V>(L)
template <int V>
__device__ __forceinline__ float2 warp_reduce_ds_t(float2* v) {
  const int lane = threadIdx.x & 31;
  int off = 16;
#pragma unroll
  for (int n = V; n > 1; n >>= 1, off >>= 1) {
    const bool hi = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < n / 2; ++i) {
      const float2 send = hi ? v[i] : v[i + n / 2];
      const float2 keep = hi ? v[i + n / 2] : v[i];
      v[i] = ds_add(keep, shfl_xor_ds(send, off));
    }
  }
  float2 t = v[0];
#pragma unroll
  for (; off > 0; off >>= 1) t = ds_add(t, shfl_xor_ds(t, off));
  return t;
}

// team_reduce_vec with double-single values and sums (same buffers, same protocol: callers
// alternate between two `mine` buffers; one cluster barrier per call on cluster teams)
__device__ void team_reduce_vec_ds(Team& tm, const float2* mine, float2* out, int nval) {
  __syncthreads();
  cg::cluster_group cl = cg::this_cluster();
  if (tm.kind == TEAM_CLUSTER) {
    cl.sync();
    for (int k = threadIdx.x; k < nval; k += NT) {
      float2 a[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) a[r] = r < tm.size ? *cl.map_shared_rank(mine + k, r) : make_float2(0.f, 0.f);
#pragma unroll
      for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
        for (int r = 0; r < w; ++r) a[r] = ds_add(a[r], a[r + w]);
      out[k] = a[0];
    }
  } else {
    const int cs = tm.csize;
    const int crank = (int)cl.block_rank();
    const int cid = tm.rank / cs;
    const int ncl = tm.size / cs;
    float2* buf = reinterpret_cast<float2*>(team_partials(tm));
    cl.sync();
    for (int k = crank * NT + threadIdx.x; k < nval; k += cs * NT) {
      float2 a[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) a[r] = r < cs ? *cl.map_shared_rank(mine + k, r) : make_float2(0.f, 0.f);
#pragma unroll
      for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
        for (int r = 0; r < w; ++r) a[r] = ds_add(a[r], a[r + w]);
      buf[(long long)cid * nval + k] = a[0];
    }
    team_sync(tm);
    for (int k = threadIdx.x; k < nval; k += NT) {
      float2 s = make_float2(0.f, 0.f);
      for (int c = 0; c < ncl; ++c) s = ds_add(s, buf[(long long)c * nval + k]);
      out[k] = s;
    }
    tm.parity ^= 1;
  }
  __syncthreads();
}

// double-single phases of the diagonal of R; the coefficients and reflector heads take the
// storage of the FP64 QR's (unused here: the kernel's static shared memory is at its limit)
__shared__ float4 s_qd_ph[TTNS_MAX_D];
struct QRDsShared {
  float4* coef;   // tau_j v_j^H W[k] of the trailing columns
  float4* vhead;  // heads of the unnormalised reflectors
  float4* ph;
};
static_assert(sizeof(double2) == sizeof(float4), "aliased QR arrays");

__device__ __noinline__ void op_qr_ds(const KernelParams& P, Team& tm, const Instr& I, double2* work) {
  QRShared& qs = s_qs;
  const QRDsShared qd = {reinterpret_cast<float4*>(qs.coef), reinterpret_cast<float4*>(qs.vhead), s_qd_ph};
  PhaseClock pc;
  pc.start(P.profile && tm.rank == 0 && threadIdx.x == 0, tm.kind == TEAM_GRID);
  const NodeDesc nd = P.nodes[I.node];
  const int l = I.leg;
  const int n = nd.dims[l];
  const long long rows = nd.size / n;
  double2* A = P.pool + nd.off;
  float4* W = reinterpret_cast<float4*>(work);  // column-major: W[c * rows + r]
  double2* Rout = P.pool + P.trees[I.tree].bond_off;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long chunk = (rows + tm.size - 1) / tm.size;
  const long long rb = min(rows, (long long)tm.rank * chunk);
  const long long re = min(rows, rb + chunk);
  const int nr = (int)(re - rb);
  const float inv_nr = nr > 0 ? 1.0f / (float)nr : 0.0f;
  // shared memory: two partial buffers and the sums (PB double-single values each), the own
  // rows of the workspace, T (FP64), the scaled T and Z (double-single), the product scratch
  const int PB = max(2 * n * n, 4 * n + 4);
  float2* red[2] = {reinterpret_cast<float2*>(dyn_smem), reinterpret_cast<float2*>(dyn_smem) + PB};
  float2* redo = red[1] + PB;
  int rp = 0;
  const long long ws_off = (3LL * PB * (long long)sizeof(float2) + 15) & ~15LL;
  const bool in_smem = ws_off + (long long)n * chunk * (long long)sizeof(float4) <= P.smem_bytes;
  float4* const Wl = in_smem ? reinterpret_cast<float4*>(dyn_smem + ws_off) : W;
  const long long ldw = in_smem ? chunk : rows;
  const long long roff = in_smem ? rb : 0;
  auto WA = [&](int c, long long r) -> float4& { return Wl[(long long)c * ldw + (r - roff)]; };
  const long long g_off = (ws_off + (in_smem ? (long long)n * chunk * (long long)sizeof(float4) : 0) + 15) & ~15LL;
  const bool g_smem = g_off + 3LL * n * n * 16 <= P.smem_bytes;
  const int ldg = g_smem ? n : TTNS_MAX_D;
  double2* Tm = g_smem ? reinterpret_cast<double2*>(dyn_smem + g_off)
                       : P.cta_scratch + (long long)blockIdx.x * P.cta_scratch_stride;
  float4* Ts = reinterpret_cast<float4*>(Tm + ldg * ldg);  // shat_j T[j][i] shat_i
  float4* Z = Ts + ldg * ldg;
  // copy into the column-major workspace; the Frobenius norm sets the null threshold
  DsAcc fro;
  fro.init(make_float2(0.f, 0.f));
  for (int idx = threadIdx.x; idx < n * nr; idx += NT) {
    const int c = fdivu(idx, nr, inv_nr);
    const long long r = rb + (idx - c * nr);
    const float4 a = ds_cfrom(A[qr_addr(nd, l, r, c)]);
    WA(c, r) = a;
    fro.mac(ds_re(a), ds_re(a));
    fro.mac(ds_im(a), ds_im(a));
  }
  __syncthreads();
  const long long p_off = (g_off + (g_smem ? 3LL * n * n * 16 : 0) + 15) & ~15LL;
  const bool p_smem = g_smem && p_off + 32LL * n * (long long)sizeof(float4) <= P.smem_bytes;
  float4* const prod = reinterpret_cast<float4*>(dyn_smem + p_off);
  // per CTA, over the own rows r > jj, for the columns c = jj .. n-1:
  //   slots 4 (c - jj) + {0, 1}: d_c = sum_r conj(W[jj][r]) W[c][r];  {2, 3}: h_c = W[c][jj]
  auto prepare = [&](int jj, float2* mine) {
    const int nc = n - jj;
    const long long r1 = max(rb, (long long)jj + 1);
    const int nrw = (int)max(0LL, re - r1);
    if (p_smem && chunk <= 32) {
      for (int idx = threadIdx.x; idx < nc * 32; idx += NT) {
        const int c = idx >> 5, rr = idx & 31;
        float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
        if (rr < nrw) {
          const long long r = r1 + rr;
          DsAcc ar, ai;
          ar.init(make_float2(0.f, 0.f));
          ai.init(make_float2(0.f, 0.f));
          ds_conj_mac(ar, ai, WA(jj, r), WA(jj + c, r));
          p = ds_c(ar.val(), ai.val());
        }
        prod[idx] = p;
      }
      __syncthreads();
      const int ntask = nc * 8;
      for (int idx = threadIdx.x; idx < ((ntask + 31) & ~31); idx += NT) {
        const bool on = idx < ntask;
        const int c = idx >> 3, g = idx & 7;
        float2 sr = make_float2(0.f, 0.f), si = sr;
        if (on) {
          const float4* pc2 = prod + c * 32 + g;
          const float4 s0 = pc2[0], s1 = pc2[8], s2 = pc2[16], s3 = pc2[24];
          sr = ds_add(ds_add(ds_re(s0), ds_re(s1)), ds_add(ds_re(s2), ds_re(s3)));
          si = ds_add(ds_add(ds_im(s0), ds_im(s1)), ds_add(ds_im(s2), ds_im(s3)));
        }
#pragma unroll
        for (int o = 4; o >= 1; o >>= 1) {
          sr = ds_add(sr, shfl_xor_ds(sr, o));
          si = ds_add(si, shfl_xor_ds(si, o));
        }
        if (on && g == 0) {
          mine[4 * c] = sr;
          mine[4 * c + 1] = si;
        }
      }
    } else {
      for (int c0 = 0; c0 < nc; c0 += 4 * NWARP) {
        DsAcc acc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q].init(make_float2(0.f, 0.f));
        for (long long r = r1 + lane; r < re; r += 32) {
          const float4 vr = WA(jj, r);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int c = c0 + warp + q * NWARP;
            if (c < nc) ds_conj_mac(acc[2 * q], acc[2 * q + 1], vr, WA(jj + c, r));
          }
        }
        float2 v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = acc[q].val();
        const float2 t = warp_reduce_ds_t<8>(v);
        if ((lane & 3) == 0) {
          const int vid = warp_reduce_vid<8>(lane);
          const int c = c0 + warp + (vid >> 1) * NWARP;
          if (c < nc) mine[4 * c + (vid & 1)] = t;
        }
      }
    }
    const bool own_row = rb <= jj && jj < re;
    for (int c = threadIdx.x; c < nc; c += NT) {
      const float4 h = own_row ? WA(jj + c, jj) : make_float4(0.f, 0.f, 0.f, 0.f);
      mine[4 * c + 2] = ds_re(h);
      mine[4 * c + 3] = ds_im(h);
    }
  };
  {
    float2* mine = red[rp];
    rp ^= 1;
    prepare(0, mine);
    __shared__ float2 s_fro[NWARP];
    float2 f = fro.val();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) f = ds_add(f, shfl_xor_ds(f, o));
    if (lane == 0) s_fro[warp] = f;
    __syncthreads();
    if (threadIdx.x == 0) {
      float2 sum = s_fro[0];
      for (int w = 1; w < NWARP; ++w) sum = ds_add(sum, s_fro[w]);
      mine[4 * n] = sum;
    }
    team_reduce_vec_ds(tm, mine, redo, 4 * n + 1);
  }
  pc.lap(P.ctl, 8);
  const double fro_m = sqrt(fmax(ds_to(redo[4 * n]), 0.0));
  const double thr = P.qr_cutoff * fro_m;
  for (int j = 0; j < n; ++j) {
    // the reflector in FP64 from the reduced sums (the same formulas as op_qr)
    const double2 x0 = make_double2(ds_to(redo[2]), ds_to(redo[3]));
    const double dj = fmax(ds_to(redo[0]), 0.0);
    const double ax2 = x0.x * x0.x + x0.y * x0.y;
    const double sigma = sqrt(ax2 + dj);
    const double ax = sqrt(ax2);
    double tau = 0.0, shat = 0.0;
    double2 vh = make_double2(0, 0), alpha = make_double2(0, 0);
    const bool null = !(sigma > thr);
    if (!null) {
      const bool head = ax > 0.0;
      const double inv_ax = head ? 1.0 / ax : 0.0;
      const double hv = ax + sigma;
      const double vn2 = dj + hv * hv;
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
      qs.rdiag[j] = alpha;
      qd.vhead[j] = ds_cfrom(vh);
    }
    if (!null && nk > 0) {
      // c_k = tau (d_k + conj(vh) h_k), in double-single
      const float4 vhd = ds_cfrom(vh);
      const float2 taud = ds_from(tau);
      for (int k = threadIdx.x; k < nk; k += NT) {
        const int sl = 4 * (k + 1);
        DsAcc ar, ai;
        ar.init(redo[sl]);
        ai.init(redo[sl + 1]);
        ds_conj_mac(ar, ai, vhd, ds_c(redo[sl + 2], redo[sl + 3]));
        DsAcc cr, ci;
        cr.init(make_float2(0.f, 0.f));
        ci.init(make_float2(0.f, 0.f));
        cr.mac(taud, ar.val());
        ci.mac(taud, ai.val());
        qd.coef[k] = ds_c(cr.val(), ci.val());
      }
      __syncthreads();
      pc.lap(P.ctl, 13);
      // W[k] -= v c_k on the own rows r >= j
      const long long r0 = max(rb, (long long)j);
      const int nrr = (int)max(0LL, re - r0);
      const float inv_nrr = nrr > 0 ? 1.0f / (float)nrr : 0.0f;
      // four elements per thread in flight (their loads issued together)
      const int tot = nk * nrr;
      for (int idx0 = threadIdx.x; idx0 < tot; idx0 += 4 * NT) {
        float4 w[4], vr[4], ck[4];
        float4* wp[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int idx = min(idx0 + u * NT, tot - 1);  // clamped: a duplicate is not stored
          const int k = fdivu(idx, nrr, inv_nrr);
          const long long r = r0 + (idx - k * nrr);
          vr[u] = (r == j) ? qd.vhead[j] : WA(j, r);
          ck[u] = qd.coef[k];
          wp[u] = &WA(j + 1 + k, r);
          w[u] = *wp[u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          DsAcc ar, ai;
          ar.init(ds_re(w[u]));
          ai.init(ds_im(w[u]));
          ds_cmac(ar, ai, make_float4(-vr[u].x, -vr[u].y, -vr[u].z, -vr[u].w), ck[u]);
          w[u] = ds_c(ar.val(), ai.val());
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (idx0 + u * NT < tot) *wp[u] = w[u];
      }
    }
    if (nk > 0) {
      __syncthreads();
      pc.lap(P.ctl, 14);
      float2* mine = red[rp];
      rp ^= 1;
      prepare(j + 1, mine);
      pc.lap(P.ctl, 15);
      team_reduce_vec_ds(tm, mine, redo, 4 * nk);
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
  // Gram of the unit reflectors over the own rows for the pairs a <= b (pair p = b (b + 1) / 2
  // + a), double-single partials, one team reduction
  const int npair = n * (n + 1) / 2;
  {
    float2* mine = red[rp];
    rp ^= 1;
    for (int p = threadIdx.x; p < npair; p += NT) {
      int b = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
      while ((b + 1) * (b + 2) / 2 <= p) ++b;
      while (b * (b + 1) / 2 > p) --b;
      const int a = p - b * (b + 1) / 2;
      DsAcc g0r, g0i, g1r, g1i;
      g0r.init(make_float2(0.f, 0.f));
      g0i.init(make_float2(0.f, 0.f));
      g1r.init(make_float2(0.f, 0.f));
      g1i.init(make_float2(0.f, 0.f));
      if (qs.tau[a] != 0.0 && qs.tau[b] != 0.0) {
        long long r = max(rb, (long long)b);
        for (; r + 1 < re; r += 2) {
          const float4 va0 = (r == a) ? qd.vhead[a] : WA(a, r);
          const float4 vb0 = (r == b) ? qd.vhead[b] : WA(b, r);
          const float4 va1 = WA(a, r + 1);
          const float4 vb1 = (r + 1 == b) ? qd.vhead[b] : WA(b, r + 1);
          ds_conj_mac(g0r, g0i, va0, vb0);
          ds_conj_mac(g1r, g1i, va1, vb1);
        }
        if (r < re) {
          const float4 va0 = (r == a) ? qd.vhead[a] : WA(a, r);
          const float4 vb0 = (r == b) ? qd.vhead[b] : WA(b, r);
          ds_conj_mac(g0r, g0i, va0, vb0);
        }
      }
      mine[2 * p] = ds_add(g0r.val(), g1r.val());
      mine[2 * p + 1] = ds_add(g0i.val(), g1i.val());
    }
    team_reduce_vec_ds(tm, mine, redo, 2 * npair);
  }
  // Gram of the unit reflectors, Gd[a][b] = shat_a shat_b (reduced sum), a <= b, double-single,
  // in the partial buffer that the last reduction's barrier released
  float4* Gd = reinterpret_cast<float4*>(red[rp]);
  for (int p = threadIdx.x; p < npair; p += NT) {
    int b = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
    while ((b + 1) * (b + 2) / 2 <= p) ++b;
    while (b * (b + 1) / 2 > p) --b;
    const int a = p - b * (b + 1) / 2;
    const float2 sab = ds_from(qs.shat[a] * qs.shat[b]);
    DsAcc gr, gi;
    gr.init(make_float2(0.f, 0.f));
    gi.init(make_float2(0.f, 0.f));
    gr.mac(sab, redo[2 * p]);
    gi.mac(sab, redo[2 * p + 1]);
    Gd[a * n + b] = ds_c(gr.val(), gi.val());
  }
  // T (upper triangular, double-single, in the storage of Tm): T[j][j] = 2, T[0:j, j] =
  // -2 T[0:j, 0:j] G[0:j, j] (rows and columns of identity reflectors stay zero); four lanes
  // per row i split the dot and add by shuffles.  Ts[i][j] = shat_i T[i][j] shat_j for Z.
  float4* Td = reinterpret_cast<float4*>(Tm);
  for (int idx = threadIdx.x; idx < n * n; idx += NT) {
    Td[idx / n * ldg + idx % n] = make_float4(0.f, 0.f, 0.f, 0.f);
    Ts[idx / n * ldg + idx % n] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();
  pc.lap(P.ctl, 10);
  {
    const int i = threadIdx.x >> 2, q = threadIdx.x & 3;
    for (int j = 0; j < n; ++j) {
      const bool tj = qs.tau[j] != 0.0;
      const bool on = tj && i < j;
      DsAcc sr, si;
      sr.init(make_float2(0.f, 0.f));
      si.init(make_float2(0.f, 0.f));
      if (on)
        for (int k = i + q; k < j; k += 4) ds_cmac(sr, si, Td[i * ldg + k], Gd[k * n + j]);
      float2 vr = sr.val(), vi = si.val();
#pragma unroll
      for (int o = 1; o <= 2; o <<= 1) {  // within the aligned group of four lanes
        vr = ds_add(vr, shfl_xor_ds(vr, o));
        vi = ds_add(vi, shfl_xor_ds(vi, o));
      }
      if (on && q == 0) {
        const float4 t = make_float4(-2.f * vr.x, -2.f * vr.y, -2.f * vi.x, -2.f * vi.y);  // exact
        Td[i * ldg + j] = t;
        const float2 sij = ds_from(qs.shat[i] * qs.shat[j]);
        DsAcc a, b;
        a.init(make_float2(0.f, 0.f));
        b.init(make_float2(0.f, 0.f));
        a.mac(sij, ds_re(t));
        b.mac(sij, ds_im(t));
        Ts[i * ldg + j] = ds_c(a.val(), b.val());
      }
      if (threadIdx.x == 0 && tj) {
        Td[j * ldg + j] = make_float4(2.f, 0.f, 0.f, 0.f);
        Ts[j * ldg + j] = ds_c(ds_from(2.0 * qs.shat[j] * qs.shat[j]), make_float2(0.f, 0.f));
      }
      __syncthreads();
    }
  }
  // Z[j][c] = sum_{j <= i <= c} Ts[j][i] conj(V[c][i]) (upper triangular), so that
  // Q = I - V Z with the unnormalised V of the workspace
  for (int idx = threadIdx.x; idx < n * n; idx += NT) {
    const int j = idx / n, c = idx % n;
    DsAcc zr, zi;
    zr.init(make_float2(0.f, 0.f));
    zi.init(make_float2(0.f, 0.f));
    for (int i = j; i <= c; ++i) {
      if (qs.tau[i] == 0.0) continue;
      const float4 t = Ts[j * ldg + i];
      const float4 v = (c == i) ? qd.vhead[i] : W[(long long)i * rows + c];
      // t conj(v)
      zr.mac(ds_re(t), ds_re(v));
      zr.mac(ds_im(t), ds_im(v));
      zi.mac(ds_im(t), ds_re(v));
      zi.mac(ds_neg(ds_re(t)), ds_im(v));
    }
    Z[j * ldg + c] = ds_c(zr.val(), zi.val());
  }
  pc.lap(P.ctl, 11);
  for (int j = threadIdx.x; j < n; j += NT) {
    const double2 a = qs.rdiag[j];
    const double aa = sqrt(a.x * a.x + a.y * a.y);
    const double2 p = aa > 0.0 ? make_double2(a.x / aa, a.y / aa) : make_double2(1.0, 0.0);
    qs.ph[j] = p;
    qd.ph[j] = ds_cfrom(p);
  }
  __syncthreads();
  // R (row j scaled by conj(ph_j)) into the bond buffer, rescaled to ||R||_F = ||M||_F
  if (tm.rank == 0) {
    __shared__ double s_rn[NWARP];
    double loc = 0.0;
    for (int idx = threadIdx.x; idx < n * n; idx += NT) {
      const int j = idx / n, k = idx % n;
      double2 r = make_double2(0, 0);
      if (k > j) r = ds_cto(W[(long long)k * rows + j]);
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
      if (k > j) r = ds_cto(W[(long long)k * rows + j]);
      else if (k == j) r = qs.rdiag[j];
      const double2 p = qs.ph[j];
      Rout[idx] = make_double2(scale * (r.x * p.x + r.y * p.y), scale * (r.y * p.x - r.x * p.y));
    }
  }
  // Q[r][c] = (delta_rc - sum_{j <= min(r, c)} V[r][j] Z[j][c]) ph_c over the own rows; a thread
  // takes the columns c0 = 2 cp and c0 + 1 of one row (V[r][j] loaded once for both; Z[j][c] = 0
  // for j > c)
  const int ncp = (n + 1) / 2;
  for (int idx = threadIdx.x; idx < ncp * nr; idx += NT) {
    const int cp = fdivu(idx, nr, inv_nr);
    const long long r = rb + (idx - cp * nr);
    const int c0 = 2 * cp, c1 = c0 + 1;
    const bool has1 = c1 < n;
    const int jmax = (int)(r < (long long)(has1 ? c1 : c0) ? r : (long long)(has1 ? c1 : c0));
    DsAcc q0r, q0i, q1r, q1i;
    q0r.init(make_float2(r == c0 ? 1.f : 0.f, 0.f));
    q0i.init(make_float2(0.f, 0.f));
    q1r.init(make_float2(r == c1 ? 1.f : 0.f, 0.f));
    q1i.init(make_float2(0.f, 0.f));
    for (int j = 0; j <= jmax; ++j) {
      if (qs.tau[j] == 0.0) continue;
      const float4 v = (r == j) ? qd.vhead[j] : WA(j, r);
      const float4 nv = make_float4(-v.x, -v.y, -v.z, -v.w);
      const float4 z0 = Z[j * ldg + c0];
      const float4 z1 = has1 ? Z[j * ldg + c1] : make_float4(0.f, 0.f, 0.f, 0.f);
      ds_cmac(q0r, q0i, nv, z0);
      ds_cmac(q1r, q1i, nv, z1);
    }
    {
      DsAcc o_r, o_i;
      o_r.init(make_float2(0.f, 0.f));
      o_i.init(make_float2(0.f, 0.f));
      ds_cmac(o_r, o_i, ds_c(q0r.val(), q0i.val()), qd.ph[c0]);
      A[qr_addr(nd, l, r, c0)] = make_double2(ds_to(o_r.val()), ds_to(o_i.val()));
    }
    if (has1) {
      DsAcc o_r, o_i;
      o_r.init(make_float2(0.f, 0.f));
      o_i.init(make_float2(0.f, 0.f));
      ds_cmac(o_r, o_i, ds_c(q1r.val(), q1i.val()), qd.ph[c1]);
      A[qr_addr(nd, l, r, c1)] = make_double2(ds_to(o_r.val()), ds_to(o_i.val()));
    }
  }
  team_sync(tm);
  pc.lap(P.ctl, 12);
}

// A_u <- R applied on leg I.leg (the gauge absorb of the mixed modes) in double-single: the
// tensor is converted once into the workspace, R into shared memory, every element is a
// compensated dot of length dims[leg], and the result is written back in FP64.
__device__ __noinline__ void op_absorb_ds(const KernelParams& P, Team& tm, const Instr& I, double2* work) {
  const NodeDesc nd = P.nodes[I.node];
  const long long N = nd.size;
  double2* A = P.pool + nd.off;
  const double2* R = P.pool + P.trees[I.tree].bond_off;
  const int l = I.leg;
  const int D = nd.dims[l];
  const int st = nd.strides[l];
  float4* Ad = reinterpret_cast<float4*>(work);
  float4* Rd = reinterpret_cast<float4*>(dyn_smem);  // D x D <= 64 KB
  for (long long idx = tm.gtid(); idx < N; idx += tm.nthr()) Ad[idx] = ds_cfrom(A[idx]);
  for (int k = threadIdx.x; k < D * D; k += NT) Rd[k] = ds_cfrom(R[k]);
  team_sync(tm);
  for (long long idx = tm.gtid(); idx < N; idx += tm.nthr()) {
    const LegPos lp = leg_pos(nd, l, idx);
    const float4* row = Rd + lp.i * D;
    const float4* xp = Ad + lp.base;
    DsAcc ar0, ai0, ar1, ai1;
    ar0.init(make_float2(0.f, 0.f));
    ai0.init(make_float2(0.f, 0.f));
    ar1.init(make_float2(0.f, 0.f));
    ai1.init(make_float2(0.f, 0.f));
    int k = 0;
    for (; k + 1 < D; k += 2) {
      ds_cmac(ar0, ai0, row[k], xp[(long long)k * st]);
      ds_cmac(ar1, ai1, row[k + 1], xp[(long long)(k + 1) * st]);
    }
    if (k < D) ds_cmac(ar0, ai0, row[k], xp[(long long)k * st]);
    const float2 r = ds_add(ar0.val(), ar1.val()), i = ds_add(ai0.val(), ai1.val());
    A[idx] = make_double2(ds_to(r), ds_to(i));
  }
  team_sync(tm);
}
