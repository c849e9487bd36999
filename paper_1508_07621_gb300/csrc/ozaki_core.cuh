// FP64 emulation of the dense Chebyshev product on the BF16 tensor cores (FQ_OZAKI): Ozaki's
// error-free splitting (Ozaki, Ogita, Oishi, Rump 2012, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its applications") with
// fixed-point BF16 slices and exact FP32 sums in tensor memory.
//
// Splitting.  Every row r of an operand (a state row of Psi, re and im together; a row of
// Omega~_m, S and A together) gets one power-of-two scale 2^e_r >= its largest entry.  x / 2^e_r
// (|x / 2^e_r| < 1/2) is rounded to 48 fractional bits as a 64-bit integer and cut into OZ_S
// signed digits of 8 bits by rounding shifts,
//   x = 2^e_r * sum_q d_q 2^(-8 (q+1)) + (remainder below 2^-49 of the scale),  |d_q| <= 128,
// each slice d_q 2^(-8(q+1)) exact in BF16 (integer work only: GB300 runs FP64 far below its
// integer and FP32 rates).  The slices of a row share one binary grid, so a product of slice a
// of the left and slice b of the right operand is an integer multiple of 2^(-8(a+b+2)) and sums
// of such products are exact in FP32 while they stay below 2^24 units.
//
// Product.  Y[j][i] = sum_k Psi[j][k] (S[i][k] + i A[i][k]) takes the 21 slice pairs (a, b) with
// a + b <= 5 (terms beyond carry less than 2^-48 of the scales).  Pairs with a + b = 0, 1, 2 go
// to three exact accumulators, the rest (a + b >= 3, at most 2^-24 of the leading term) to a
// fourth one whose FP32 rounding stays near 2^-48 relative.  Per 128 values of k the four
// accumulators are drained into double-float registers (an FP32 pair, about 48 bits) by the
// epilogue warps: over 128 values of k (256 products per pair) the worst exact sum is
// 3 pairs * 2^14 * 256 < 2^24 units.  The
// complex product uses three right-operand blocks per row block, [-A; S; A]: Psi_r . [S; A]^T
// and Psi_i . [-A; S]^T accumulate Yr and Yi side by side, two MMAs of N = 128 per pair.
//
// Chain (Eqs. 10-12).  States stay FP64 in HBM; the epilogue applies the recurrence, the Bessel
// accumulation and the step phase in FP64, as the plain FP64 path does.  A separate pass slices
// each new Psi_{l+1} (its row scales need the whole row).
//
// Kernel.  One 128-state x 64-column tile per CTA: warp 0 streams TMA stages (K = 16 per stage,
// 32-byte rows with 32-byte swizzle), warp 1 issues the MMAs, warps 2-17 drain tensor memory
// (four warps per lane quarter, 16 complex columns each).  The 512 tensor-memory columns hold
// the four accumulators (128 columns each), so the MMAs wait for each drain.  Every wait is
// bounded; a wait that gives up records FQ_BIT_TIMEOUT, drains this CTA's own copies and MMAs,
// frees tensor memory and returns.
#pragma once

#include "split_core.cuh"

namespace {

constexpr int OZ_S = 6;                     // slices per operand
constexpr int OZ_PAIRS = OZ_S * (OZ_S + 1) / 2;
constexpr int OZ_BN = 64;                   // complex output columns per tile
constexpr int OZ_ROWB = 32;                 // bytes per K row of a stage (K = 16 BF16)
constexpr int OZ_BKE = OZ_ROWB / 2;
constexpr int OZ_KB_PER_DRAIN = 8;          // 128 values of k between drains
constexpr int OZ_EPI_WARPS = 16;
constexpr int OZ_THREADS = 64 + 32 * OZ_EPI_WARPS;
constexpr int OZ_A_BYTES = BM * OZ_ROWB;                   // one slice of Psi_r or Psi_i
constexpr uint32_t OZ_TMEM_COLS = 512;      // 4 accumulators x (Yr | Yi) x 64 columns
constexpr int OZ_XS_BYTES = 64 * 4 * 32 * OZ_EPI_WARPS;   // drained sums staged for the epilogue

// Stage layout of the complex product (Omega~ = S + i A): one right slice is the [-A; S; A] rows
// of a 64-row block.  (Products with a real right operand use ozaki_real.cuh.)
struct OzCfg {
  static constexpr int R_ROWS = 3 * OZ_BN;
  static constexpr int R_BYTES = R_ROWS * OZ_ROWB;
  static constexpr int STAGE_BYTES = 2 * OZ_S * OZ_A_BYTES + OZ_S * R_BYTES;
  static constexpr int STAGES = 2;
  static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 1024 + 256;
  static_assert((size_t)STAGES * STAGE_BYTES >= OZ_XS_BYTES + 16 * sizeof(double2), "epilogue staging");
};

struct OzMaps {
  CUtensorMap a[OZ_S];  // left slices [rows][2 np]: Psi_r in columns [0, np), Psi_i in [np, 2 np)
  CUtensorMap r[OZ_S];  // right slices: [3 np][np] (per 64-row block of Omega~, rows -A, S, A), or
                        // [np][np] for a real operator (ozaki_real.cuh)
};

// Epilogue of one product Y = Psi . Omega~^T (FP64 states, row stride n):
enum OzMode {
  OZ_FWD = 0,  // Chebyshev term: psi_{l+1} = -2i Y + psi_{l-1}, acc += a psi_{l+1}, phase at the last term
  OZ_ADJ = 1,  // adjoint term: out = cpa g + i cw Y + b2
  OZ_DOT = 2,  // gradient dot: partial[cta] = sum over the tile of conj(b) Y
};

struct OzEpi {
  int n, nc;
  const double* cur_re;   // FWD: psi_l (first term: psi_0); ADJ: g; DOT: b
  const double* cur_im;
  const double* prev_re;  // FWD: psi_{l-1}; ADJ: b2 (NULL: absent)
  const double* prev_im;
  double* acc_re;
  double* acc_im;
  double* out_re;         // FWD: psi_{l+1} (in place of psi_{l-1}) or X at the last term; ADJ: out
  double* out_im;
  const int* es;          // row exponents of the left slices
  const int* et;          // row exponents of the right slices
  double cpa_re, cpa_im, cw;  // ADJ coefficients
  double2* partial;       // DOT: one per CTA
  fq_term t;
};

// K-major 32-byte rows with 32-byte swizzle, 8-row atoms of 256 bytes
__device__ __forceinline__ uint64_t oz_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)((8 * OZ_ROWB) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)6 << 61;
  return d;
}

// pair p -> (a, b), ordered by a + b, then a
__device__ __forceinline__ void oz_pair(int p, int& a, int& b) {
  int d = 0, base = 0;
  while (p >= base + d + 1) {
    base += d + 1;
    ++d;
  }
  a = p - base;
  b = d - a;
}

__device__ __forceinline__ float2 neg2f(float2 a) { return make_float2(-a.x, -a.y); }

// (h, l) += v in double-float for two values at once (packed FP32x2): Knuth's two-sum, then a
// fast renormalisation; explicitly rounded operations only
__device__ __forceinline__ void dd_add2(float2& h, float2& l, float2 v) {
  const float2 s = __fadd2_rn(h, v);
  const float2 bb = __fadd2_rn(s, neg2f(h));
  const float2 e = __fadd2_rn(__fadd2_rn(h, neg2f(__fadd2_rn(s, neg2f(bb)))), __fadd2_rn(v, neg2f(bb)));
  const float2 lo = __fadd2_rn(l, e);
  const float2 h2 = __fadd2_rn(s, lo);
  l = __fadd2_rn(lo, neg2f(__fadd2_rn(h2, neg2f(s))));
  h = h2;
}

__device__ __forceinline__ double pow2(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

// |x| as an ordered integer key (the bit pattern of a non-negative double orders like its value)
__device__ __forceinline__ unsigned long long abs_key(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// row exponent E with |x| < 2^(E-1) for the row maximum (key of |max|; 0 for a zero row):
// E = (unbiased exponent of max) + 2, kept in the normal range
__device__ __forceinline__ int oz_exponent(unsigned long long key) {
  if (key == 0) return 0;
  const int be = (int)(key >> 52);  // biased exponent (subnormals: 0)
  const int e = be - 1023 + 2;
  return e < -960 ? -960 : e;
}

// Slices of a 48-bit fixed-point value R = r 2^48 (|r| < 1/2): signed 8-bit digits d_q by
// rounding shifts, slice q = d_q 2^(-8(q+1)) in BF16 (exact: |d_q| <= 128).
__device__ __forceinline__ void oz_digits_fixed(long long R, __nv_bfloat16 (&s)[OZ_S]) {
#pragma unroll
  for (int q = 0; q < OZ_S; ++q) {
    const int sh = 40 - 8 * q;
    long long d;
    if (sh > 0) {
      d = (R + (1ll << (sh - 1))) >> sh;
      R -= d << sh;
    } else {
      d = R;
    }
    s[q] = __float2bfloat16_rn((float)(int)d * __int_as_float((127 - 8 * (q + 1)) << 23));
  }
}

// The digits of r = x / 2^E (|r| < 1/2): R = r 2^48 rounded to an integer, then d_q by rounding
// shifts of 8 bits; slices d_q 2^(-8(q+1)) in BF16.  R comes straight from the bit pattern of x
// (x = m 2^(b - 1075) with the 53-bit significand m and biased exponent b, so R = m shifted right
// by 1027 + E - b >= 6 bits, rounded half away from zero): integer work only.
__device__ __forceinline__ void oz_digits(double x, int E, __nv_bfloat16 (&s)[OZ_S]) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int b = (int)((bits >> 52) & 0x7FF);
  const int sh = 1027 + E - b;
  long long R = 0;
  if (b != 0 && sh < 64) {  // zero and subnormal entries (below 2^-1022) give zero digits
    const unsigned long long m = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    R = (long long)((m + (1ull << (sh - 1))) >> sh);
    if (bits >> 63) R = -R;
  }
  oz_digits_fixed(R, s);
}

__device__ __forceinline__ unsigned long long block_max_key(unsigned long long v, unsigned long long* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  unsigned long long m = 0;
  for (int q = 0; q < nw; ++q) m = red[q] > m ? red[q] : m;
  __syncthreads();
  return m;
}

// Left slices of the state rows v = c x (x = the FP64 rows re, im; NULL: identity rows), with an
// optional FP64 copy of v: one CTA per row j of the padded block (rows >= nc are zero).
__device__ __forceinline__ void oz_row_value(const double* re, const double* im, double cr, double ci, int n, int j,
                                             int k, double& vr, double& vi) {
  double a, b;
  if (re) {
    a = re[(size_t)j * n + k];
    b = im[(size_t)j * n + k];
  } else {
    a = j == k ? 1.0 : 0.0;
    b = 0.0;
  }
  if (ci == 0.0 && cr == 1.0) {  // plain slicing: no FP64 arithmetic
    vr = a;
    vi = b;
  } else {
    vr = cr * a - ci * b;
    vi = cr * b + ci * a;
  }
}

__device__ __forceinline__ uint2 pack4(__nv_bfloat16 a, __nv_bfloat16 b, __nv_bfloat16 c, __nv_bfloat16 d) {
  return make_uint2((uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16),
                    (uint32_t)__bfloat16_as_ushort(c) | ((uint32_t)__bfloat16_as_ushort(d) << 16));
}

__global__ void k_oz_slice_left(const double* __restrict__ re, const double* __restrict__ im, double cr, double ci,
                                double* __restrict__ out_re, double* __restrict__ out_im, int n, int nc, int np,
                                size_t astride, __nv_bfloat16* __restrict__ left, int* __restrict__ es) {
  __shared__ unsigned long long red[32];
  const int j = blockIdx.x;
  unsigned long long m = 0;
  if (j < nc)
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      double vr, vi;
      oz_row_value(re, im, cr, ci, n, j, k, vr, vi);
      if (out_re) {
        out_re[(size_t)j * n + k] = vr;
        out_im[(size_t)j * n + k] = vi;
      }
      const unsigned long long a = abs_key(vr), b = abs_key(vi);
      m = a > m ? a : m;
      m = b > m ? b : m;
    }
  const int e = oz_exponent(block_max_key(m, red));
  __nv_bfloat16* row = left + (size_t)j * 2 * np;
  // four consecutive columns per thread: one 8-byte store per slice and part (np % 4 == 0, and
  // every slice row starts on an 8-byte boundary)
  for (int k0 = 4 * threadIdx.x; k0 < np; k0 += 4 * blockDim.x) {
    __nv_bfloat16 sr[4][OZ_S], si[4][OZ_S];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      double xr = 0.0, xi = 0.0;
      if (j < nc && k0 + u < n) oz_row_value(re, im, cr, ci, n, j, k0 + u, xr, xi);
      oz_digits(xr, e, sr[u]);
      oz_digits(xi, e, si[u]);
    }
#pragma unroll
    for (int q = 0; q < OZ_S; ++q) {
      *reinterpret_cast<uint2*>(row + q * astride + k0) = pack4(sr[0][q], sr[1][q], sr[2][q], sr[3][q]);
      *reinterpret_cast<uint2*>(row + q * astride + np + k0) = pack4(si[0][q], si[1][q], si[2][q], si[3][q]);
    }
  }
  if (threadIdx.x == 0) es[j] = e;
}

// Omega~_m = sum_t c_t M_t - sbeta 1 split into S (symmetric terms) and A (antisymmetric ones).
struct OzOmega {
  const double* m[FQ_M6_TERMS];
  double c[FQ_M6_TERMS];
  int anti[FQ_M6_TERMS];
  int terms;
  double sbeta;
};

__device__ __forceinline__ void oz_omega_entry(const OzOmega& a, int n, int i, int k, double& S, double& A) {
  S = i == k ? -a.sbeta : 0.0;
  A = 0.0;
  const size_t o = (size_t)i * n + k;
  for (int t = 0; t < a.terms; ++t) {
    if (a.anti[t]) A = fma(a.c[t], a.m[t][o], A);
    else S = fma(a.c[t], a.m[t][o], S);
  }
}

// Right slices of step m: one CTA per row i of the padded operator (rows >= n are zero).
__global__ void k_oz_omega(const __grid_constant__ OzOmega a, int n, int np, size_t rstride,
                           __nv_bfloat16* __restrict__ right, int* __restrict__ et) {
  __shared__ unsigned long long red[32];
  const int i = blockIdx.x;
  unsigned long long m = 0;
  if (i < n)
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      double S, A;
      oz_omega_entry(a, n, i, k, S, A);
      const unsigned long long x = abs_key(S), y = abs_key(A);
      m = x > m ? x : m;
      m = y > m ? y : m;
    }
  const int e = oz_exponent(block_max_key(m, red));
  const size_t rb = (size_t)(3 * OZ_BN) * (i / OZ_BN) + (i % OZ_BN);  // row of -A; S and A follow
  for (int k = threadIdx.x; k < np; k += blockDim.x) {
    double S = 0.0, A = 0.0;
    if (i < n && k < n) oz_omega_entry(a, n, i, k, S, A);
    __nv_bfloat16 ss[OZ_S], sa[OZ_S];
    oz_digits(S, e, ss);
    oz_digits(A, e, sa);
#pragma unroll
    for (int q = 0; q < OZ_S; ++q) {
      __nv_bfloat16* base = right + q * rstride + k;
      base[rb * np] = __hneg(sa[q]);
      base[(rb + OZ_BN) * np] = ss[q];
      base[(rb + 2 * OZ_BN) * np] = sa[q];
    }
  }
  if (threadIdx.x == 0) et[i] = e;
}

// Slices of the real operator v = ((h0 ? h0 : 0) + c1 h1) inv - shift 1, c1 = f[m] (1 without f):
// one CTA per row i of [np][np] (rows >= n are zero).  The adjoint's Omega~_m (piecewise-constant
// drive) and E = H1 / Delta E.
__device__ __forceinline__ double oz_real_entry(const double* h0, const double* h1, double c1, double inv,
                                                double shift, int n, int i, int k) {
  const size_t o = (size_t)i * n + k;
  return ((h0 ? h0[o] : 0.0) + c1 * h1[o]) * inv - (i == k ? shift : 0.0);
}

__global__ void k_oz_real(const double* __restrict__ h0, const double* __restrict__ h1, const double* __restrict__ f,
                          int m, double inv, double shift, int n, int np, size_t rstride,
                          __nv_bfloat16* __restrict__ right, int* __restrict__ et) {
  __shared__ unsigned long long red[32];
  const int i = blockIdx.x;
  const double c1 = f ? f[m] : 1.0;
  unsigned long long mx = 0;
  if (i < n)
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const unsigned long long a = abs_key(oz_real_entry(h0, h1, c1, inv, shift, n, i, k));
      mx = a > mx ? a : mx;
    }
  const int e = oz_exponent(block_max_key(mx, red));
  for (int k0 = 4 * threadIdx.x; k0 < np; k0 += 4 * blockDim.x) {
    __nv_bfloat16 sl[4][OZ_S];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const double v = (i < n && k0 + u < n) ? oz_real_entry(h0, h1, c1, inv, shift, n, i, k0 + u) : 0.0;
      oz_digits(v, e, sl[u]);
    }
#pragma unroll
    for (int q = 0; q < OZ_S; ++q)
      *reinterpret_cast<uint2*>(right + q * rstride + (size_t)i * np + k0) = pack4(sl[0][q], sl[1][q], sl[2][q], sl[3][q]);
  }
  if (threadIdx.x == 0) et[i] = e;
}

// One Chebyshev term (OZ_FWD) on a 128-state x 64-column tile (see the file comment).
__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_oz_term(const __grid_constant__ OzMaps maps, int nk, int tiles_j, int tiles_i, int np, OzEpi e) {
  using Cfg = OzCfg;
  constexpr int OZ_STAGES = Cfg::STAGES;
  constexpr int OZ_STAGE_BYTES = Cfg::STAGE_BYTES;
  constexpr int OZ_R_BYTES = Cfg::R_BYTES;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = smem_raw + (base - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + OZ_STAGES * OZ_STAGE_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * OZ_STAGES + 6);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + OZ_STAGES);
  // tempty0 + 8 g: accumulator g of the last chunk is drained (the drain warps release them one by one)
  const uint32_t tfull = smem_u32(bars + 2 * OZ_STAGES), tempty0 = smem_u32(bars + 2 * OZ_STAGES + 1);
  const uint32_t done = smem_u32(bars + 2 * OZ_STAGES + 5);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchunks = nk / OZ_KB_PER_DRAIN;

  int tj, ti;
  {
    const int b = blockIdx.x, per = RASTER_GROUP * tiles_i, g = b / per;
    const int gj = min(RASTER_GROUP, tiles_j - g * RASTER_GROUP), r = b - g * per;
    tj = g * RASTER_GROUP + r % gj;
    ti = r / gj;
  }
  const int j0 = tj * BM, i0 = ti * OZ_BN;

  if (threadIdx.x == 0) {
    for (int s = 0; s < OZ_STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(tfull, 1);
    for (int g = 0; g < 4; ++g) mbar_init(tempty0 + 8 * g, OZ_EPI_WARPS);
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(OZ_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {  // ---------------- TMA producer
      int issued = 0;
      bool ok = true;
      for (int kb = 0; kb < nk && ok; ++kb) {
        const int s = kb % OZ_STAGES;
        if (kb >= OZ_STAGES && !(ok = mbar_wait(empty0 + 8 * s, ((kb / OZ_STAGES) - 1) & 1))) break;
        if (*(volatile int*)abort_flag) {
          ok = false;
          break;
        }
        const uint32_t st = base + s * OZ_STAGE_BYTES;
        const uint32_t bar = full0 + 8 * s;
        mbar_expect_tx(bar, OZ_STAGE_BYTES);
        const int kx = kb * OZ_BKE;
#pragma unroll
        for (int q = 0; q < OZ_S; ++q) {
          tma_load_2d(st + (2 * q) * OZ_A_BYTES, &maps.a[q], bar, kx, j0);           // Psi_r
          tma_load_2d(st + (2 * q + 1) * OZ_A_BYTES, &maps.a[q], bar, np + kx, j0);  // Psi_i
          tma_load_2d(st + 2 * OZ_S * OZ_A_BYTES + q * OZ_R_BYTES, &maps.r[q], bar, kx, 3 * i0);  // -A, S, A
        }
        issued = kb + 1;
      }
      if (!ok) {
        atomicExch(abort_flag, 1);
        atomicOr(e.t.status, FQ_BIT_TIMEOUT);
      }
      for (int kb = max(0, issued - OZ_STAGES); kb < issued; ++kb)
        mbar_wait(full0 + 8 * (kb % OZ_STAGES), (kb / OZ_STAGES) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ---------------- MMA issuer
      constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)((2 * OZ_BN) >> 3) << 17) |
                                 ((uint32_t)(BM >> 4) << 24);
      bool ok = true;
      int kb = 0;
      for (int c = 0; c < nchunks && ok; ++c) {
        for (int kq = 0; kq < OZ_KB_PER_DRAIN && ok; ++kq, ++kb) {
          const int s = kb % OZ_STAGES;
          ok = mbar_wait(full0 + 8 * s, (kb / OZ_STAGES) & 1);
          if (!ok || *(volatile int*)abort_flag) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = base + s * OZ_STAGE_BYTES;
          // descriptors of the stage's tiles: the start-address field is the low 14 bits (16-byte
          // units), so an offset inside shared memory adds to the descriptor without a carry
          const uint64_t d0 = oz_desc(st);
          // the pairs in descending order, accumulator 3 (15 pairs) first: at a chunk's first stage
          // each accumulator's MMAs wait only for that accumulator's drain, so the later ones drain
          // while accumulator 3's MMAs run
#pragma unroll
          for (int p = OZ_PAIRS - 1; p >= 0; --p) {
            int a, b;
            oz_pair(p, a, b);
            const int g = a + b < 3 ? a + b : 3;
            const bool lead = p == 20 || p == 5 || p == 2 || p == 0;  // first pair of each accumulator
            if (kq == 0 && lead && c > 0) {
              if (!(ok = mbar_wait(tempty0 + 8 * g, (c - 1) & 1))) break;
              tc_fence_after();
            }
            const uint32_t acc = tmem + (uint32_t)g * (2 * OZ_BN);
            const uint32_t rb = 2 * OZ_S * OZ_A_BYTES + b * OZ_R_BYTES;
            const uint32_t first = (kq == 0 && lead) ? 0u : 1u;
            mma_bf16(acc, d0 + (uint64_t)(((2 * a) * OZ_A_BYTES) >> 4), d0 + (uint64_t)((rb + OZ_BN * OZ_ROWB) >> 4),
                     idesc, first);  // Psi_r . [S; A]
            mma_bf16(acc, d0 + (uint64_t)(((2 * a + 1) * OZ_A_BYTES) >> 4), d0 + (uint64_t)(rb >> 4), idesc,
                     1u);            // Psi_i . [-A; S]
          }
          mma_commit(empty0 + 8 * s);
        }
        if (!ok) break;
        mma_commit(tfull);
      }
      if (!ok) {
        atomicExch(abort_flag, 1);
        atomicOr(e.t.status, FQ_BIT_TIMEOUT);
      }
      mma_commit(done);
      mbar_wait(done, 0);
    }
  } else {  // ---------------- drain warps 2-17
    const int quarter = warp & 3, part = (warp - 2) >> 2;
    const int j = j0 + quarter * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(part * 16);
    float2 hr[8], lr[8], hi[8], li[8];  // double-float sums of columns (2p, 2p + 1)
#pragma unroll
    for (int q = 0; q < 8; ++q) hr[q] = lr[q] = hi[q] = li[q] = make_float2(0.f, 0.f);
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      bool go = mbar_wait(tfull, c & 1);
      tc_fence_after();
      go = __all_sync(0xffffffffu, go && !*(volatile int*)abort_flag);
      if (!go) {
        ok = false;
        break;
      }
      // one 16-column load at a time keeps the double-float sums and one load in registers;
      // accumulator 3 first (the next chunk's MMAs start with it), each released once read
#pragma unroll
      for (int g = 3; g >= 0; --g) {
#pragma unroll
        for (int part_im = 0; part_im < 2; ++part_im) {
          float v[16];
          tmem_ld16(trow + g * (2 * OZ_BN) + part_im * OZ_BN, v);
          tmem_wait_ld();
          float2* h = part_im ? hi : hr;
          float2* l = part_im ? li : lr;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float2 w = make_float2(v[2 * q], v[2 * q + 1]);
            if (g < 3) dd_add2(h[q], l[q], w);
            else l[q] = __fadd2_rn(l[q], w);  // below 2^-24 of the leading sum: the low word carries it
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty0 + 8 * g);  // the next chunk's MMAs into it may start
      }
    }
    if (!ok) {
      atomicExch(abort_flag, 1);
      atomicOr(e.t.status, FQ_BIT_TIMEOUT);
    } else if (j < e.nc) {
      // ---------------- epilogue in FP64 (as in the plain FP64 path).  The stages are idle now
      // (the last MMAs have completed): the sums wait there, one column per pass.
      float* xs = reinterpret_cast<float*>(gbase) + (threadIdx.x - 64);
      constexpr int XS = 32 * OZ_EPI_WARPS;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        xs[(8 * q) * XS] = hr[q].x;
        xs[(8 * q + 1) * XS] = lr[q].x;
        xs[(8 * q + 2) * XS] = hi[q].x;
        xs[(8 * q + 3) * XS] = li[q].x;
        xs[(8 * q + 4) * XS] = hr[q].y;
        xs[(8 * q + 5) * XS] = lr[q].y;
        xs[(8 * q + 6) * XS] = hi[q].y;
        xs[(8 * q + 7) * XS] = li[q].y;
      }
      const fq_term& t = e.t;
      const int ej = e.es[j];
      bool bad = false;
#pragma unroll 1
      for (int q = 0; q < 16; ++q) {
        const int i = i0 + part * 16 + q;
        if (i >= e.n) break;
        const int ex = ej + e.et[i];
        const double sc = pow2(ex < -1022 ? -1022 : ex);  // below that the product is below 2^-1022
        const int b = 8 * (q >> 1) + 4 * (q & 1);  // slots of column q: hr, lr, hi, li
        const double yr = ((double)xs[b * XS] + (double)xs[(b + 1) * XS]) * sc;
        const double yi = ((double)xs[(b + 2) * XS] + (double)xs[(b + 3) * XS]) * sc;
        const size_t idx = (size_t)j * e.n + i;
        double pr, pi;
        if (t.first) {
          pr = yi;
          pi = -yr;
        } else {
          pr = fma(2.0, yi, e.prev_re[idx]);
          pi = fma(-2.0, yr, e.prev_im[idx]);
        }
        bad |= !(pr * pr + pi * pi <= t.bound2);
        double ar, ai;
        if (t.first) {
          ar = fma(t.coef, pr, t.coef0 * e.cur_re[idx]);
          ai = fma(t.coef, pi, t.coef0 * e.cur_im[idx]);
        } else {
          ar = fma(t.coef, pr, e.acc_re[idx]);
          ai = fma(t.coef, pi, e.acc_im[idx]);
        }
        if (t.last) {
          e.out_re[idx] = t.ph_re * ar - t.ph_im * ai;
          e.out_im[idx] = t.ph_re * ai + t.ph_im * ar;
        } else {
          e.out_re[idx] = pr;
          e.out_im[idx] = pi;
          e.acc_re[idx] = ar;
          e.acc_im[idx] = ai;
        }
      }
      if (bad) atomicOr(t.status, FQ_BIT_BOUND);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS) : "memory");
  }
}


}  // namespace
