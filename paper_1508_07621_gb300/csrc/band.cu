// The tridiagonal chain as one banded product per step on the tensor cores, in FP64 emulation
// (FQ_OZAKI with a tridiagonal plan).
//
// Step m applies X_m = P_m X_{m-1} with P_m = e^{-i beta h} sum_k c_k T_k(Omega~_m), c_k =
// (-i)^k a_k (Eqs. 10 and 12).  Omega~_m is tridiagonal, so T_k(Omega~_m) has bandwidth k and the
// step's whole polynomial is a band matrix with 2L + 1 diagonals.  Instead of L sparse products on
// every state, each step
//   1. forms the rows of P_m once (k_band_rows): in the real gauge frame Omega~ = D Omega' D^+
//      (gauge.cuh), row i of P(Omega') is P(Omega') e_i (P(Omega') is complex symmetric), computed
//      by Clenshaw's recurrence in double-float arithmetic on a 96-row window around i, which holds
//      its support i +- L; then P_m[i][k] = e^{-i beta h} e^{i theta_i} v_k e^{-i theta_k} in FP64;
//   2. multiplies every state, held as fixed-point BF16 slices (as FQ_OZAKI does for dense
//      operators, ozaki_core.cuh), by the band on the tensor cores (k_oz_band): a tile of 64
//      operator rows [i0, i0 + 64) needs only the state columns [i0 - kh, i0 + 64 + kh) (kh = L
//      rounded up to 8), so its K loop is that window instead of all N columns.  The 21 slice
//      pairs sum exactly in FP32 tensor memory over the whole window (3 pairs x 2^14 x 320
//      products < 2^24 units), so one drain per tile suffices; the epilogue forms the new states
//      as double-float pairs with FP32 instructions only (GB300's FP64 rate is far below its FP32
//      and tensor rates) and cuts them into the next step's slices at a predicted scale;
//   3. fixes the scales and cuts again any state that outgrew its prediction (k_band_fixup).
// Between steps the slices are the states; the double-float states are written at the last step
// (and for single entries the slices cannot hold).  A call's input states are sliced once
// (k_band_rowmax, k_band_slice).
// The product is the same polynomial the Chebyshev recurrence applies, so the result agrees with
// the plain chain to the emulation's rounding (48 bits per slice product).  Needs L <= 47.
//
// Layouts (all in the caller's workspace).  Both operands of the product are stored MN-major (the
// states, or the operator rows, contiguous; K the outer index), so that every row of a TMA box is
// 64 BF16 = 128 bytes (128-byte swizzle) although a K stage is only 16 deep: the K-major form
// (16 BF16 = 32-byte box rows) fed the tensor cores at about two thirds of the rate.
//   states     double-float [nc][npl] float4 (re_hi, re_lo, im_hi, im_lo), npl = N rounded to 128
//              (the input, the output, and entries the slices cannot hold)
//   left       OZ_S slices [2 npl][ncp] BF16: row k the real parts of component k of every
//              state, row npl + k the imaginary parts
//   right      OZ_S slices [nrows / 64][kw][192] BF16: per 64-row block b and window column
//              c = k - (64 b - kh) the columns -Im, Re, Im of rows 64 b .. 64 b + 63 of P_m
//   cf, rot    per step (2 d, 2 e') and (cos, sin) theta of the gauge frame, FP64, [nsteps][nrows]
#include <atomic>

#include "gauge.cuh"
#include "ozaki_core.cuh"

namespace {

constexpr int BAND_LANE_ROWS = 3;                       // window rows per lane
constexpr int BAND_WIN = 32 * BAND_LANE_ROWS;           // 96-row window, centre at position 48
constexpr int BAND_MAXL = BAND_WIN / 2 - 1;             // support i +- L inside the window
constexpr int BAND_KH = 48;                             // widest K half-width of a 64-row block's window
constexpr int BAND_KW = OZ_BN + 2 * BAND_KH;            // at most 160 columns of K per tile (10 stages)
constexpr int BAND_ROWS_PER_CTA = 8;                    // one warp per operator row
static_assert(BAND_KH >= BAND_MAXL, "the K window covers every row's band");
static_assert(3LL * (1 << 14) * (2 * BAND_KW) < (1LL << 24), "one drain per tile keeps the exact sums exact");

struct BandCoef {
  dfl c[BAND_MAXL + 1];  // c_k = c[k] for even k, i c[k] for odd k
};

__device__ __forceinline__ dflc shfl_dflc(dflc a, int delta, bool up) {
  dflc r;
  if (up) {
    r.h.x = __shfl_up_sync(0xffffffffu, a.h.x, delta);
    r.h.y = __shfl_up_sync(0xffffffffu, a.h.y, delta);
    r.l.x = __shfl_up_sync(0xffffffffu, a.l.x, delta);
    r.l.y = __shfl_up_sync(0xffffffffu, a.l.y, delta);
  } else {
    r.h.x = __shfl_down_sync(0xffffffffu, a.h.x, delta);
    r.h.y = __shfl_down_sync(0xffffffffu, a.h.y, delta);
    r.l.x = __shfl_down_sync(0xffffffffu, a.l.x, delta);
    r.l.y = __shfl_down_sync(0xffffffffu, a.l.y, delta);
  }
  return r;
}

// One Clenshaw update on the lane's three window rows: out = (2 Omega' x) - out (HALF: the
// closing Omega' x - out), plus c_k at the centre row (c = cc or i cc for IM), double-float.
template <bool IM, bool HALF>
__device__ __forceinline__ void band_apply(const dflc (&x)[BAND_LANE_ROWS], dflc (&out)[BAND_LANE_ROWS],
                                           const dfl (&d)[BAND_LANE_ROWS], const dfl (&e)[BAND_LANE_ROWS], dfl el0,
                                           dfl cc, int lane) {
  const dflc z = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  dflc left = shfl_dflc(x[BAND_LANE_ROWS - 1], 1, true);
  dflc right = shfl_dflc(x[0], 1, false);
  if (lane == 0) left = z;    // beyond the window: never reached by the support (L <= 47)
  if (lane == 31) right = z;
#pragma unroll
  for (int q = 0; q < BAND_LANE_ROWS; ++q) {
    const dflc xm = q == 0 ? left : x[q - 1];
    const dflc xp = q == BAND_LANE_ROWS - 1 ? right : x[q + 1];
    dfl dq = d[q], el = q == 0 ? el0 : e[q - 1], eh = e[q];
    if (HALF) {  // the stored operator is 2 Omega'; halving is exact
      dq = {0.5f * dq.h, 0.5f * dq.l};
      el = {0.5f * el.h, 0.5f * el.l};
      eh = {0.5f * eh.h, 0.5f * eh.l};
    }
    dflc acc = dflc_fma(dq, x[q], dflc_fma(el, xm, dflc_fma(eh, xp, dflc_neg(out[q]))));
    if (q == 0 && lane == BAND_WIN / 2 / BAND_LANE_ROWS) {  // centre row: + c_k e_i
      const dflc c = IM ? dflc{make_float2(0.f, cc.h), make_float2(0.f, cc.l)}
                        : dflc{make_float2(cc.h, 0.f), make_float2(cc.l, 0.f)};
      acc = dflc_add(acc, c);
    }
    out[q] = acc;
  }
}

// What one step's band formation needs: the step's gauge tables (row k of cf, rot), the band
// slices and row exponents it writes, and the tile geometry (kh, a multiple of 8 in [L, 48], is
// the K half-width of the product's tile windows: a tile row holds 64 + 2 kh columns).
struct BandRows {
  const double2* cf;
  const double2* rot;
  __nv_bfloat16* right;
  int* et;
  size_t rstride;
  double ph_re, ph_im;
  int n, nrows, L, kh;
};

typedef __nv_bfloat16 BandStage[3][BAND_KW][BAND_ROWS_PER_CTA];  // one slice's staged 8-row block

// One warp forms row i < nrows of P_m (zero for i >= n) into column r8 of the staged 8-row block
// of the right operand slices, and its exponent et[i].
__device__ __forceinline__ void band_form_row(const BandRows& a, const BandCoef& coef, int i, int r8,
                                              BandStage* stage, int lane) {
  const int n = a.n, L = a.L, kh = a.kh;
  const double2* __restrict__ cf = a.cf;
  const double2* __restrict__ rot = a.rot;
  const bool live = i < n;
  const int w0 = i - BAND_WIN / 2;  // row of window position 0
  const dfl zd = {0.f, 0.f};
  const dflc zc = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  dfl d[BAND_LANE_ROWS], e[BAND_LANE_ROWS];
  dflc A[BAND_LANE_ROWS], B[BAND_LANE_ROWS];
#pragma unroll
  for (int q = 0; q < BAND_LANE_ROWS; ++q) {
    const int k = w0 + BAND_LANE_ROWS * lane + q;
    if (live && k >= 0 && k < n) {
      const double2 c = cf[k];
      d[q] = dfl_of(c.x);
      e[q] = dfl_of(c.y);  // 2 Omega'[k+1][k] (0 for the last row)
    } else {
      d[q] = zd;
      e[q] = zd;
    }
    A[q] = zc;
    B[q] = zc;
  }
  dfl el0;
  el0.h = __shfl_up_sync(0xffffffffu, e[BAND_LANE_ROWS - 1].h, 1);
  el0.l = __shfl_up_sync(0xffffffffu, e[BAND_LANE_ROWS - 1].l, 1);
  if (lane == 0) el0 = (live && w0 >= 1 && w0 - 1 < n) ? dfl_of(cf[w0 - 1].y) : zd;

  if (live) {
    // b_L = c_L e_i, b_{L+1} = 0; then b_k = c_k e_i + 2 Omega' b_{k+1} - b_{k+2}
    if (lane == BAND_WIN / 2 / BAND_LANE_ROWS) {
      const dfl cL = coef.c[L];
      A[0] = (L & 1) ? dflc{make_float2(0.f, cL.h), make_float2(0.f, cL.l)}
                     : dflc{make_float2(cL.h, 0.f), make_float2(cL.l, 0.f)};
    }
    int k = L - 1;
    while (k >= 2) {
      if (k & 1) band_apply<true, false>(A, B, d, e, el0, coef.c[k], lane);
      else band_apply<false, false>(A, B, d, e, el0, coef.c[k], lane);
      --k;
      if (k & 1) band_apply<true, false>(B, A, d, e, el0, coef.c[k], lane);
      else band_apply<false, false>(B, A, d, e, el0, coef.c[k], lane);
      --k;
    }
    if (k == 1) {  // b_1 into B, then the sum c_0 e_i + Omega' b_1 - b_2 into A
      band_apply<true, false>(A, B, d, e, el0, coef.c[1], lane);
      band_apply<false, true>(B, A, d, e, el0, coef.c[0], lane);
    } else {  // b_1 in A, b_2 in B: the sum into B, then moved to A
      band_apply<false, true>(A, B, d, e, el0, coef.c[0], lane);
#pragma unroll
      for (int q = 0; q < BAND_LANE_ROWS; ++q) A[q] = B[q];
    }
  }
  // P_m[i][k] = e^{-i beta h} e^{i theta_i} v_k e^{-i theta_k} in FP64, and the row's scale
  double vr[BAND_LANE_ROWS], vi[BAND_LANE_ROWS];
  unsigned long long key = 0;
  const double2 ri = live ? rot[i] : make_double2(1.0, 0.0);
  const double wr = a.ph_re * ri.x - a.ph_im * ri.y, wi = a.ph_re * ri.y + a.ph_im * ri.x;  // e^{-i beta h} e^{i theta_i}
#pragma unroll
  for (int q = 0; q < BAND_LANE_ROWS; ++q) {
    const int k = w0 + BAND_LANE_ROWS * lane + q;
    vr[q] = vi[q] = 0.0;
    if (live && k >= 0 && k < n) {
      const double2 rk = rot[k];
      const double ur = wr * rk.x + wi * rk.y, ui = wi * rk.x - wr * rk.y;  // times e^{-i theta_k}
      const double sr = (double)A[q].h.x + (double)A[q].l.x, si = (double)A[q].h.y + (double)A[q].l.y;
      vr[q] = ur * sr - ui * si;
      vi[q] = ur * si + ui * sr;
    }
    const unsigned long long a = abs_key(vr[q]), b = abs_key(vi[q]);
    key = a > key ? a : key;
    key = b > key ? b : key;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, key, o);
    key = w > key ? w : key;
  }
  const int E = oz_exponent(key);
  const int r = i % OZ_BN;
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
  // window positions [p0, p1) (the row's band; L <= kh) go to tile columns c = r + p - 48 + kh
  const int kw = OZ_BN + 2 * kh;
  const int p0 = BAND_WIN / 2 - kh > 0 ? BAND_WIN / 2 - kh : 0;
  const int p1 = BAND_WIN / 2 + kh + 1 < BAND_WIN ? BAND_WIN / 2 + kh + 1 : BAND_WIN;
#pragma unroll
  for (int q = 0; q < BAND_LANE_ROWS; ++q) {
    const int pos = BAND_LANE_ROWS * lane + q;
    if (pos < p0 || pos >= p1) continue;
    __nv_bfloat16 sr[OZ_S], si[OZ_S];
    oz_digits(vr[q], E, sr);
    oz_digits(vi[q], E, si);
    const int c = r + pos - BAND_WIN / 2 + kh;
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) {
      stage[s][0][c][r8] = __hneg(si[s]);
      stage[s][1][c][r8] = sr[s];
      stage[s][2][c][r8] = si[s];
    }
  }
  // the row's other columns of the tile window: [0, r) and [r + p1 - p0, kw)
  const int bw = p1 - p0, nz = kw - bw;
#pragma unroll
  for (int zz = 0; zz < 2; ++zz) {
    const int z = lane + 32 * zz;
    if (z >= nz) continue;
    const int c = z < r ? z : z + bw;
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) {
      stage[s][0][c][r8] = zero;
      stage[s][1][c][r8] = zero;
      stage[s][2][c][r8] = zero;
    }
  }
  if (lane == 0) a.et[i] = E;
}

// The staged block of rows 8 b8 .. 8 b8 + 7 to the MN-major band: column c of part (-Im, Re, Im)
// of 64-row block b, rows r0 .. r0 + 7, at [(b kw + c) 192 + 64 part + r0] as one 16-byte piece;
// thread t of nt.
__device__ __forceinline__ void band_store_block(const BandRows& a, int b8, const BandStage* stage, int t, int nt) {
  const int kw = OZ_BN + 2 * a.kh;
  const int i0 = b8 * BAND_ROWS_PER_CTA, b = i0 / OZ_BN, r0 = i0 % OZ_BN;
  for (int x = t; x < OZ_S * 3 * kw; x += nt) {
    const int c = x % kw, sp = x / kw, part = sp % 3, s = sp / 3;
    *reinterpret_cast<uint4*>(a.right + s * a.rstride + ((size_t)b * kw + c) * (3 * OZ_BN) + part * OZ_BN + r0) =
        *reinterpret_cast<const uint4*>(&stage[s][part][c][0]);
  }
}

// Rows i < nrows of P_m (the first step of a call; later steps' bands are formed inside the
// previous step's product, k_oz_band): one warp per row, 8 rows per CTA (nrows is a multiple of
// 64, so the grid holds no partial CTA and a CTA's rows share one 64-row block), staged in shared
// memory and written as 16-byte pieces of the MN-major band.
__global__ void __launch_bounds__(32 * BAND_ROWS_PER_CTA) k_band_rows(const BandRows a, const BandCoef coef) {
  __shared__ __align__(16) BandStage stage[OZ_S];
  const int lane = threadIdx.x & 31, r8 = threadIdx.x >> 5;
  band_form_row(a, coef, blockIdx.x * BAND_ROWS_PER_CTA + r8, r8, stage, lane);
  __syncthreads();
  band_store_block(a, blockIdx.x, stage, threadIdx.x, blockDim.x);
}

// float 2^e for |e| <= 126 (clamped)
__device__ __forceinline__ float pow2f(int e) {
  e = e < -126 ? -126 : (e > 127 ? 127 : e);
  return __int_as_float((127 + e) << 23);
}

__device__ __forceinline__ void two_sum2(float2& a, float2& b) {  // (a, b) <- (fl(a + b), its error), exact
  const float2 s = __fadd2_rn(a, b);
  const float2 bb = __fadd2_rn(s, neg2f(a));
  b = __fadd2_rn(__fadd2_rn(a, neg2f(__fadd2_rn(s, neg2f(bb)))), __fadd2_rn(b, neg2f(bb)));
  a = s;
}

// The OZ_S slices of v = a + b (a double-float pair, packed as (re, im), |v| < 1/2 in units of
// the row scale), with FP32 instructions only: t_q = v rounded to a multiple of 2^(-8(q+1)) by
// adding and subtracting 1.5 2^(15 - 8q) (exact for |v| < 2^(14 - 8q)), then v -= t_q (exact) and a
// two-sum keeps the remainder as a normalised pair.  t_q = d_q 2^(-8(q+1)) with |d_q| <= 128 (a
// remainder is at most half a grid step), exact in BF16; the part below 2^-49 is dropped.
// Returns |t_0| <= 1/2 for both parts (false: the value broke the scale bound).
__device__ __forceinline__ bool df_digits2(float2 a, float2 b, __nv_bfloat16 (&dr)[OZ_S], __nv_bfloat16 (&di)[OZ_S]) {
  two_sum2(a, b);
  bool ok = true;
#pragma unroll
  for (int q = 0; q < OZ_S; ++q) {
    const float c = __int_as_float((127 + 15 - 8 * q) << 23) * 1.5f;
    const float2 t = __fadd2_rn(__fadd2_rn(a, make_float2(c, c)), make_float2(-c, -c));
    if (q == 0) ok = fabsf(t.x) <= 0.5f && fabsf(t.y) <= 0.5f;
    dr[q] = __float2bfloat16_rn(t.x);
    di[q] = __float2bfloat16_rn(t.y);
    a = __fadd2_rn(a, neg2f(t));
    two_sum2(a, b);
  }
  return ok;
}

// A state's slice exponent from its largest |hi| part (an FP32 bit pattern, 0 for a zero state):
// E = exponent + 2, so every |X[j][k]| < 2^(E-1) with a factor 2 to spare, below 1/2 in units of
// the scale 2^E.
__device__ __forceinline__ int band_key_exp(unsigned int key) { return key == 0u ? 0 : (int)(key >> 23) - 127 + 2; }

// The product's epilogue cuts X_m into the next step's slices before X_m's maxima are known, at
// the exponent of X_{m-1}'s maximum plus this margin: a state then fits unless its maximum grows
// by more than 2^BAND_MARGIN (between 2 and 4 times) in one step.  A margin of 0 flagged so many
// states (any growth across a power of 2) that cutting them again cost more than the slicing
// pass it replaces; 1 costs one bit of the 48 on the states' scale.
constexpr int BAND_MARGIN = 1;

// Each state's largest |hi| part (re or im) as an FP32 key, for the slicing of states that no
// product has written yet (the first step of a call); one CTA per state j < nc.
__global__ void k_band_rowmax(const float4* __restrict__ x, int n, int ld, unsigned int* __restrict__ kmax) {
  __shared__ unsigned long long red[32];
  const int j = blockIdx.x;
  unsigned long long m = 0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const float4 v = x[(size_t)j * ld + k];
    const unsigned long long a = __float_as_uint(v.x) & 0x7FFFFFFFu, b = __float_as_uint(v.z) & 0x7FFFFFFFu;
    m = a > m ? a : m;
    m = b > m ? b : m;
  }
  m = block_max_key(m, red);
  if (threadIdx.x == 0) kmax[j] = (unsigned int)m;
}

// Left slices of the double-float states (the first step of a call; later steps' slices come from
// the product's epilogue), MN-major: slice q row k holds digit q of Re X[j][k] for every state j
// (row npl + k: Im), each state at the scale 2^E_j of band_key_exp(kmax[j]); digits by the FP32
// cut of df_digits2.  Each thread cuts a 2 x 2 block (states j, j + 1; components k,
// k + 1), so that a warp writes 128 contiguous bytes (64 states) of each slice row; states >= nc
// and components >= n are zero.  Grid (ncp / 64, npl / 16), 256 threads.
__global__ void __launch_bounds__(256)
    k_band_slice(const float4* __restrict__ x, int n, int ld, int nc, int npl, int ncp, size_t astride,
                 __nv_bfloat16* __restrict__ left, int* __restrict__ es, const unsigned int* __restrict__ kmax) {
  const int j = 2 * (blockIdx.x * 32 + (threadIdx.x & 31));
  const int k = 2 * (blockIdx.y * 8 + (threadIdx.x >> 5));
  int E[2];
  float so[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    E[u] = band_key_exp(j + u < nc ? kmax[j + u] : 0u);
    so[u] = pow2f(-E[u]);  // into units of the state's scale (exact)
  }
  if (blockIdx.y == 0 && threadIdx.x < 32) {
    es[j] = E[0];
    es[j + 1] = E[1];
  }
  __nv_bfloat16 dr[2][2][OZ_S], di[2][2][OZ_S];  // [state][component][slice]
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
      if (j + u < nc && k + v < n) a = x[(size_t)(j + u) * ld + k + v];
      df_digits2(make_float2(a.x * so[u], a.z * so[u]), make_float2(a.y * so[u], a.w * so[u]), dr[u][v], di[u][v]);
    }
#pragma unroll
  for (int q = 0; q < OZ_S; ++q)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      __nv_bfloat16* col = left + q * astride + j;
      *reinterpret_cast<__nv_bfloat162*>(col + (size_t)(k + v) * ncp) = __halves2bfloat162(dr[0][v][q], dr[1][v][q]);
      *reinterpret_cast<__nv_bfloat162*>(col + (size_t)(npl + k + v) * ncp) =
          __halves2bfloat162(di[0][v][q], di[1][v][q]);
    }
}

// After the product of a step: the scales of its slices of X_m (es_next: the predicted one of
// each state, or, for a state the product flagged because an element outgrew that scale, the exact
// one of the row maximum the product collected, knew) and the flagged states' slices cut again at
// that scale; clears the flags, and X_{m-1}'s row maxima (kprev) for the next product to fill.  A flagged state's entries come back from its slices at the
// predicted scale (the six digits' sum is exact in FP64), or, for an entry marked by a NaN leading
// digit, from the double-float value the product stored for it.  One warp per state of the padded
// block (256 threads, ncp / 8 CTAs).
__global__ void __launch_bounds__(256)
    k_band_fixup(const float4* __restrict__ x, int n, int ld, int nc, int npl, int ncp, size_t astride,
                 __nv_bfloat16* __restrict__ lnext, int* __restrict__ es_next, unsigned int* __restrict__ kprev,
                 const unsigned int* __restrict__ knew, int* __restrict__ ovf) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (j >= ncp) return;  // whole warp (no barrier below)
  const bool redo = j < nc && ovf[j] != 0;
  const int E = redo ? band_key_exp(knew[j]) : (j < nc ? band_key_exp(kprev[j]) + BAND_MARGIN : 0);
  const double sp = ldexp(1.0, j < nc ? band_key_exp(kprev[j]) + BAND_MARGIN : 0);  // the scale the product cut at
  __syncwarp();
  if (lane == 0) {
    es_next[j] = E;
    kprev[j] = 0u;
  }
  if (!redo) return;
  const float so = pow2f(-E);
  for (int k = lane; k < n; k += 32) {
    float4 v;
    __nv_bfloat16 dr[OZ_S], di[OZ_S];
#pragma unroll
    for (int q = 0; q < OZ_S; ++q) {
      dr[q] = lnext[q * astride + (size_t)k * ncp + j];
      di[q] = lnext[q * astride + (size_t)(npl + k) * ncp + j];
    }
    if (__hisnan(dr[0]) || __hisnan(di[0])) {
      v = x[(size_t)j * ld + k];
    } else {
      double re = 0.0, im = 0.0;
#pragma unroll
      for (int q = 0; q < OZ_S; ++q) {
        re += (double)__bfloat162float(dr[q]);
        im += (double)__bfloat162float(di[q]);
      }
      re *= sp;
      im *= sp;
      const float rh = (float)re, ih = (float)im;
      v = make_float4(rh, (float)(re - (double)rh), ih, (float)(im - (double)ih));
    }
    df_digits2(make_float2(v.x * so, v.z * so), make_float2(v.y * so, v.w * so), dr, di);
#pragma unroll
    for (int q = 0; q < OZ_S; ++q) {
      lnext[q * astride + (size_t)k * ncp + j] = dr[q];
      lnext[q * astride + (size_t)(npl + k) * ncp + j] = di[q];
    }
  }
  __syncwarp();
  if (lane == 0) ovf[j] = 0;
}

constexpr int BAND_RG = 16;  // state blocks per raster group

// Shared-memory descriptor of an MN-major operand with 128-byte swizzle, as the TMA boxes of
// k_oz_band lay it out: 64-element atoms (128-byte rows, 8 K rows = 1 KB) at 2 KB steps along M or
// N (one 16-row box each), the two 8-row K groups of a stage 1 KB apart.
__device__ __forceinline__ uint64_t band_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(2048 >> 4) << 16;  // leading offset: next 64-element atom along M or N
  d |= (uint64_t)(1024 >> 4) << 32;  // stride offset: next 8 rows along K
  d |= (uint64_t)1 << 46;            // descriptor version for tcgen05
  d |= (uint64_t)2 << 61;            // 128-byte swizzle
  return d;
}

struct BandEpi {
  float4* out;     // X_m, double-float [nc][ld]
  unsigned int* kmax;  // per row of X_m: largest |hi| of re or im as an FP32 key (atomicMax)
  const int* es;   // row exponents of the left slices
  const int* et;   // row exponents of the right slices
  __nv_bfloat16* lnext;       // the left slices of X_m for the next step (MN-major, as k_band_slice)
  const unsigned int* kprev;  // row maxima of X_{m-1}: the predicted scales of X_m's slices
  int* ovf;                   // per state: an element outgrew the predicted scale (set to 1)
  size_t astride;
  int write_states;           // 1: write every entry of X_m (the last step); else only entries the slices cannot hold
  int n, nc, ld, npl, ncp;
  float bound2;
  unsigned int* status;
};

// The banded product X_m[j][i] = sum_{k in window(i)} X_{m-1}[j][k] P_m[i][k] on 128-state x
// 64-row tiles, persistent: one CTA per SM walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// rasterized in groups of 16 state blocks that sweep the operator blocks together (co-running CTAs
// share each operator block and the sliding state windows in L2).  Warp 0 streams
// TMA stages (K = 16 each, 128-byte MN-major box rows), warp 1 issues the MMAs of the 21 slice
// pairs into the four accumulators (512 tensor-memory columns), warps 2-17 drain them once per
// tile into double-float registers, release the tensor memory and write the tile's slices for the
// next step (and, at the last step, its double-float states) while the next tile's MMAs run.  Every wait is bounded; a wait that gives up records FQ_BIT_TIMEOUT, drains this CTA's own
// copies and MMAs, frees tensor memory and returns.
constexpr int BAND_FORM_WARPS = 2;                             // warps 18, 19 form the next step's band
constexpr int BAND_THREADS = OZ_THREADS + 32 * BAND_FORM_WARPS;  // 20 warps x 96 registers: 5 per SM sub-partition
// Forming the next band inside the product pays once the product outlasts it: with two warps per
// SM the formation takes about a third of a 10001-state product at dim 10001, and both scale with
// the band's rows, so the rule is a number of states.
constexpr int BAND_FORM_MIN_STATES = 4096;
constexpr size_t BAND_SMEM = OzCfg::SMEM + OZ_S * sizeof(BandStage);
static_assert(BAND_SMEM <= 232448, "stages and the band staging fit the 227 KB of shared memory a CTA may use");

__global__ void __launch_bounds__(BAND_THREADS, 1)
    k_oz_band(const __grid_constant__ OzMaps maps, int tiles_j, int tiles_i, int npl, int kh, BandEpi e,
              const __grid_constant__ BandRows next, const __grid_constant__ BandCoef coef, int form_next) {
  using Cfg = OzCfg;
  constexpr int STAGES = Cfg::STAGES;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = smem_raw + (base - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + STAGES * Cfg::STAGE_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 6);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  BandStage* rstage = reinterpret_cast<BandStage*>(gbase + STAGES * Cfg::STAGE_BYTES + 256);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES);
  // tempty0 + 8 g: accumulator g of the last tile is drained (the epilogue releases them one by one)
  const uint32_t tfull = smem_u32(bars + 2 * STAGES), tempty0 = smem_u32(bars + 2 * STAGES + 1);
  const uint32_t done = smem_u32(bars + 2 * STAGES + 5);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = tiles_i * tiles_j;
  const int nk = (OZ_BN + 2 * kh) / OZ_BKE;  // K stages of the tile window
  auto coords = [&](int t, int& j0, int& i0) {
    const int per = BAND_RG * tiles_i, g = t / per;
    const int gj = min(BAND_RG, tiles_j - g * BAND_RG), r = t - g * per;
    j0 = (g * BAND_RG + r % gj) * BM;
    i0 = (r / gj) * OZ_BN;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
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
      int g = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        int j0, i0;
        coords(t, j0, i0);
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = g % STAGES;
          if (g >= STAGES && !(ok = mbar_wait(empty0 + 8 * s, ((g / STAGES) - 1) & 1))) break;
          if (*(volatile int*)abort_flag) {
            ok = false;
            break;
          }
          const uint32_t st = base + s * Cfg::STAGE_BYTES;
          const uint32_t bar = full0 + 8 * s;
          mbar_expect_tx(bar, Cfg::STAGE_BYTES);
          const int kx = i0 - kh + kb * OZ_BKE;  // K row of the states (any row); negative at the first block
          const int kr = (i0 / OZ_BN) * (OZ_BN + 2 * kh) + kb * OZ_BKE;  // K row of the band block
#pragma unroll
          for (int q = 0; q < OZ_S; ++q) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {  // states j0 + 64 h .. + 63: 2 KB boxes of 16 K rows
              tma_load_2d(st + (2 * q) * OZ_A_BYTES + 2048 * h, &maps.a[q], bar, j0 + 64 * h, kx);        // re
              tma_load_2d(st + (2 * q + 1) * OZ_A_BYTES + 2048 * h, &maps.a[q], bar, j0 + 64 * h, npl + kx);  // im
            }
#pragma unroll
            for (int c = 0; c < 3; ++c)  // band columns -Im, Re, Im
              tma_load_2d(st + 2 * OZ_S * OZ_A_BYTES + q * Cfg::R_BYTES + 2048 * c, &maps.r[q], bar, 64 * c, kr);
          }
        }
      }
      if (!ok) {
        atomicExch(abort_flag, 1);
        atomicOr(e.status, FQ_BIT_TIMEOUT);
      }
      for (int q = max(0, g - STAGES); q < g; ++q) mbar_wait(full0 + 8 * (q % STAGES), (q / STAGES) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ---------------- MMA issuer
      // FP32 accumulate, BF16 A and B, both MN-major (bits 15 and 16), N = 128, M = 128
      constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                                 ((uint32_t)((2 * OZ_BN) >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
      int g = 0, it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++it) {
        for (int kb = 0; kb < nk && ok; ++kb, ++g) {
          const int s = g % STAGES;
          ok = mbar_wait(full0 + 8 * s, (g / STAGES) & 1);
          if (!ok || *(volatile int*)abort_flag) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = base + s * Cfg::STAGE_BYTES;
          const uint64_t d0 = band_desc(st);
          // the pairs in descending order, accumulator 3 (15 pairs) first: at a tile's first stage
          // each accumulator's MMAs wait only for that accumulator's drain, so the later ones drain
          // while accumulator 3's MMAs run
#pragma unroll
          for (int p = OZ_PAIRS - 1; p >= 0; --p) {
            int a, b;
            oz_pair(p, a, b);
            const int grp = a + b < 3 ? a + b : 3;
            const bool lead = p == 20 || p == 5 || p == 2 || p == 0;  // first pair of each accumulator
            if (kb == 0 && lead && it > 0) {
              if (!(ok = mbar_wait(tempty0 + 8 * grp, (it - 1) & 1))) break;
              tc_fence_after();
            }
            const uint32_t acc = tmem + (uint32_t)grp * (2 * OZ_BN);
            const uint32_t rb = 2 * OZ_S * OZ_A_BYTES + b * Cfg::R_BYTES;
            const uint32_t first = (kb == 0 && lead) ? 0u : 1u;
            mma_bf16(acc, d0 + (uint64_t)(((2 * a) * OZ_A_BYTES) >> 4), d0 + (uint64_t)((rb + 2048) >> 4), idesc,
                     first);  // re . [Re, Im] (band boxes 1, 2)
            mma_bf16(acc, d0 + (uint64_t)(((2 * a + 1) * OZ_A_BYTES) >> 4), d0 + (uint64_t)(rb >> 4), idesc,
                     1u);     // im . [-Im, Re] (band boxes 0, 1)
          }
          mma_commit(empty0 + 8 * s);
        }
        if (!ok) break;
        mma_commit(tfull);
      }
      if (!ok) {
        atomicExch(abort_flag, 1);
        atomicOr(e.status, FQ_BIT_TIMEOUT);
      }
      mma_commit(done);
      mbar_wait(done, 0);
    }
  } else if (warp >= OZ_THREADS / 32) {  // ---------------- the next step's band, in 8-row blocks
    const int fw = warp - OZ_THREADS / 32, ft = threadIdx.x - OZ_THREADS;
    if (form_next)
      for (int b8 = blockIdx.x; b8 < next.nrows / BAND_ROWS_PER_CTA; b8 += gridDim.x) {
        for (int r8 = fw; r8 < BAND_ROWS_PER_CTA; r8 += BAND_FORM_WARPS)
          band_form_row(next, coef, b8 * BAND_ROWS_PER_CTA + r8, r8, rstage, lane);
        asm volatile("bar.sync 1, %0;" ::"n"(32 * BAND_FORM_WARPS) : "memory");  // the block is staged
        band_store_block(next, b8, rstage, ft, 32 * BAND_FORM_WARPS);
        asm volatile("bar.sync 1, %0;" ::"n"(32 * BAND_FORM_WARPS) : "memory");  // and written: reuse it
      }
  } else {  // ---------------- drain and epilogue warps 2-17
    const int quarter = warp & 3, part = (warp - 2) >> 2;
    const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(part * 16);
    bool bad = false, ok = true;
    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      int j0, i0;
        coords(t, j0, i0);
      bool go = mbar_wait(tfull, it & 1);
      tc_fence_after();
      go = __all_sync(0xffffffffu, go && !*(volatile int*)abort_flag);
      if (!go) {
        ok = false;
        break;
      }
      float2 hr[8], lr[8], hi[8], li[8];  // double-float sums of columns (2p, 2p + 1)
#pragma unroll
      for (int q = 0; q < 8; ++q) hr[q] = lr[q] = hi[q] = li[q] = make_float2(0.f, 0.f);
      // accumulator 3 first (the MMAs of the next tile start with it), each released once read
#pragma unroll
      for (int grp = 3; grp >= 0; --grp) {
#pragma unroll
        for (int part_im = 0; part_im < 2; ++part_im) {
          float v[16];
          tmem_ld16(trow + grp * (2 * OZ_BN) + part_im * OZ_BN, v);
          tmem_wait_ld();
          float2* h = part_im ? hi : hr;
          float2* l = part_im ? li : lr;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float2 w = make_float2(v[2 * q], v[2 * q + 1]);
            if (grp < 3) dd_add2(h[q], l[q], w);
            else l[q] = w;  // below 2^-24 of the leading sum: the low word carries it
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty0 + 8 * grp);  // the next tile's MMAs into it may start
      }
      const int j = j0 + quarter * 32 + lane;
      if (j < e.nc) {
        const int ej = e.es[j];
        float4* orow = e.out + (size_t)j * e.ld;
        unsigned int kmx = 0u;
        // the next step's slices of X_m at the scale X_{m-1}'s maximum predicts (the fixup pass
        // cuts a state again if an element does not fit); a warp's lanes write 32 consecutive states
        const float so = pow2f(-band_key_exp(e.kprev[j]) - BAND_MARGIN);
        __nv_bfloat16* lcol = e.lnext + j;
        bool fit = true;
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int i = i0 + part * 16 + c;
          if (i < e.n) {
            int ex = ej + e.et[i];
            ex = ex < -126 ? -126 : (ex > 127 ? 127 : ex);
            const float sc = __int_as_float((127 + ex) << 23);
            const float2 H = hr[c >> 1], Lr = lr[c >> 1], Hi = hi[c >> 1], Li = li[c >> 1];
            const float rh0 = ((c & 1) ? H.y : H.x) * sc, rl0 = ((c & 1) ? Lr.y : Lr.x) * sc;
            const float ih0 = ((c & 1) ? Hi.y : Hi.x) * sc, il0 = ((c & 1) ? Li.y : Li.x) * sc;
            const float rh = __fadd_rn(rh0, rl0), ih = __fadd_rn(ih0, il0);  // renormalise the pairs
            const float rl = __fsub_rn(rl0, __fsub_rn(rh, rh0)), il = __fsub_rn(il0, __fsub_rn(ih, ih0));
            bad |= !(rh * rh + ih * ih <= e.bound2);
            const unsigned int kr = __float_as_uint(rh) & 0x7FFFFFFFu, ki = __float_as_uint(ih) & 0x7FFFFFFFu;
            kmx = kr > kmx ? kr : kmx;
            kmx = ki > kmx ? ki : kmx;
            __nv_bfloat16 dr[OZ_S], di[OZ_S];
            const bool f = df_digits2(make_float2(rh * so, ih * so), make_float2(rl * so, il * so), dr, di);
            // between steps the slices carry the state; an entry they cannot hold is kept whole,
            // and its NaN leading digits send the fixup pass to it
            if (e.write_states || !f) orow[i] = make_float4(rh, rl, ih, il);
            if (!f) dr[0] = di[0] = __ushort_as_bfloat16((unsigned short)0x7FC0);
            fit &= f;
#pragma unroll
            for (int q = 0; q < OZ_S; ++q) {
              lcol[q * e.astride + (size_t)i * e.ncp] = dr[q];
              lcol[q * e.astride + (size_t)(e.npl + i) * e.ncp] = di[q];
            }
          }
        }
        atomicMax(e.kmax + j, kmx);
        if (!fit) e.ovf[j] = 1;
      }
    }
    if (!ok) {
      atomicExch(abort_flag, 1);
      atomicOr(e.status, FQ_BIT_TIMEOUT);
    }
    if (bad) atomicOr(e.status, FQ_BIT_BOUND);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS) : "memory");
  }
}

// complex128 rows (or the identity when x0 is NULL) into double-float rows [nc][ld], zero beyond n
__global__ void k_band_load(const double2* __restrict__ x0, float4* __restrict__ x, int nc, int n, int ld) {
  const size_t total = (size_t)nc * ld;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(q / ld), k = (int)(q % ld);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (k < n) {
      if (x0) {
        const double2 a = x0[(size_t)r * n + k];
        const dfl re = dfl_of(a.x), im = dfl_of(a.y);
        v = make_float4(re.h, re.l, im.h, im.l);
      } else if (k == r) {
        v.x = 1.f;
      }
    }
    x[q] = v;
  }
}

// double-float rows into complex128 rows [nc][n]
__global__ void k_band_store(const float4* __restrict__ x, double2* __restrict__ out, int nc, int n, int ld) {
  const size_t total = (size_t)nc * n;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(q / n), k = (int)(q % n);
    const float4 v = x[(size_t)r * ld + k];
    out[q] = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
  }
}

// U[i][j] = X_j[i] (the n x n block of states as rows -> U_T), 32 x 32 tiles through shared memory
__global__ void k_band_store_t(const float4* __restrict__ x, double2* __restrict__ u, int n, int ld) {
  __shared__ double2 tile[32][33];
  const int j0 = blockIdx.y * 32, i0 = blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int j = j0 + r, i = i0 + threadIdx.x;
    if (j < n && i < n) {
      const float4 v = x[(size_t)j * ld + i];
      tile[r][threadIdx.x] = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
    }
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = i0 + r, j = j0 + threadIdx.x;
    if (i < n && j < n) u[(size_t)i * n + j] = tile[threadIdx.x][r];
  }
}

struct BandWs {
  double2* cf;
  double2* rot;
  __nv_bfloat16* right[2];  // the band a product reads and the one it forms for the next step
  int* et[2];
  __nv_bfloat16* left[2];  // slices of the states a product reads (alternating per step)
  int* es[2];
  int* ovf;
  unsigned int* kmax[2];  // row maxima of the states a product writes (alternating per step)
  float4* x[2];
  int nrows, npl, ncp, kh, kw;
  size_t rstride, astride;
};

size_t up256b(size_t v) { return (v + 255) & ~(size_t)255; }

size_t band_layout(const fq_plan* p, int nc, int nsteps, void* base, BandWs* out) {
  BandWs w{};
  w.nrows = (p->n + OZ_BN - 1) / OZ_BN * OZ_BN;
  w.npl = (p->n + 127) & ~127;
  w.ncp = (nc + BM - 1) / BM * BM;
  // the narrowest window that holds the band with a width of whole 16-row K stages (K is the outer
  // coordinate of the MN-major boxes, so the window may start on any row)
  w.kh = std::min(BAND_KH, (p->L + 7) / 8 * 8);
  w.kw = OZ_BN + 2 * w.kh;
  w.rstride = (size_t)3 * w.nrows * w.kw;
  w.astride = (size_t)w.ncp * 2 * w.npl;
  char* b = (char*)base;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* q = b ? b + off : nullptr;
    off += up256b(bytes);
    return q;
  };
  w.cf = (double2*)take(sizeof(double2) * (size_t)nsteps * w.nrows);
  w.rot = (double2*)take(sizeof(double2) * (size_t)nsteps * w.nrows);
  for (int q = 0; q < 2; ++q) w.right[q] = (__nv_bfloat16*)take(sizeof(__nv_bfloat16) * OZ_S * w.rstride);
  for (int q = 0; q < 2; ++q) w.et[q] = (int*)take(sizeof(int) * w.nrows);
  for (int q = 0; q < 2; ++q) w.left[q] = (__nv_bfloat16*)take(sizeof(__nv_bfloat16) * OZ_S * w.astride);
  for (int q = 0; q < 2; ++q) w.es[q] = (int*)take(sizeof(int) * w.ncp);
  w.ovf = (int*)take(sizeof(int) * w.ncp);
  for (int q = 0; q < 2; ++q) w.kmax[q] = (unsigned int*)take(sizeof(unsigned int) * w.ncp);
  for (int q = 0; q < 2; ++q) w.x[q] = (float4*)take(sizeof(float4) * (size_t)nc * w.npl);
  if (out) *out = w;
  return off;
}

int band_grid(size_t total) { return (int)std::min<size_t>(std::max<size_t>((total + 255) / 256, 1), 152 * 32); }

}  // namespace

int fq_band_supported(int L) { return L >= 1 && L <= BAND_MAXL; }

size_t fq_band_workspace(const fq_plan* p, int nc, int nsteps) { return band_layout(p, nc, nsteps, nullptr, nullptr); }

fq_status fq_band_propagate(fq_plan* p, const double* x0, double* x, int nc, int m_begin, int m_end, int identity,
                            int transpose_out, void* ws, cudaStream_t s) {
  fq_status st = encode_fn();
  if (st != FQ_OK) return st;
  const int n = p->n, L = p->L, nsteps = m_end - m_begin;
  if (!fq_band_supported(L)) {
    fq_set_error("band kernel needs L <= %d (L = %d)", BAND_MAXL, L);
    return FQ_EUNSUPPORTED;
  }
  BandWs w;
  band_layout(p, nc, nsteps, ws, &w);
  OzMaps maps[2];  // per step parity: the state slices and the band a product reads
  for (int b = 0; b < 2; ++b)
    for (int q = 0; q < OZ_S; ++q) {
      // MN-major: 64-element (128-byte) box rows, 16 K rows per box
      if ((st = make_map(&maps[b].a[q], w.left[b] + q * w.astride, 2 * w.npl, w.ncp, OZ_BKE, 64)) != FQ_OK) return st;
      if ((st = make_map(&maps[b].r[q], w.right[b] + q * w.rstride, (w.nrows / OZ_BN) * w.kw, 3 * OZ_BN, OZ_BKE, 64)) !=
          FQ_OK)
        return st;
    }
  static std::atomic<unsigned> attr_set{0};
  if (fq_first_on_device(attr_set)) {
    cudaError_t e = cudaFuncSetAttribute(k_oz_band, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BAND_SMEM);
    if (e != cudaSuccess) return fq_cuda_fail(e, "band kernel shared-memory attribute");
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
  if (sms < 1) sms = 152;
  // component rows >= n of the second slice buffer stay zero (the epilogue writes rows < n only;
  // the first step's slicing pass fills the first buffer whole); no state is flagged yet, and the
  // row maxima the first product collects start at zero (the fixup pass clears them after that)
  cudaError_t ce = cudaMemsetAsync(w.ovf, 0, sizeof(int) * w.ncp, s);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(w.kmax[0], 0, sizeof(unsigned int) * w.ncp, s);
  if (nsteps > 1 && w.npl > n)
    for (int q = 0; q < OZ_S && ce == cudaSuccess; ++q)
      for (int part = 0; part < 2 && ce == cudaSuccess; ++part)
        ce = cudaMemsetAsync(w.left[1] + q * w.astride + (size_t)(part * w.npl + n) * w.ncp, 0,
                             sizeof(__nv_bfloat16) * (size_t)(w.npl - n) * w.ncp, s);
  if (ce != cudaSuccess) return fq_cuda_fail(ce, "band workspace clear");
  GaugeArgs ga{p->n, p->steps, p->d_h0, p->d_h0o, p->d_h1, p->d_k, p->d_scal, p->sbeta};
  k_gauge_tile<double><<<nsteps, GAUGE_NT, 0, s>>>(ga, w.nrows, m_begin, w.cf, w.rot);
  k_band_load<<<band_grid((size_t)nc * w.npl), 256, 0, s>>>(identity ? nullptr : (const double2*)x0, w.x[0], nc, n,
                                                            w.npl);
  BandCoef coef{};
  for (int k = 0; k <= L; ++k) {
    const double a = p->cheb[k];
    const double c = (k & 3) == 0 || (k & 3) == 3 ? a : -a;  // c_k = (-i)^k a_k: c or i c
    const float h = (float)c;
    coef.c[k] = {h, (float)(c - (double)h)};
  }
  const int tiles_i = (n + OZ_BN - 1) / OZ_BN, tiles_j = w.ncp / BM;
  const int ntiles = tiles_i * tiles_j;
  BandEpi e{};
  e.ovf = w.ovf;
  e.astride = w.astride;
  e.n = n;
  e.nc = nc;
  e.ld = w.npl;
  e.npl = w.npl;
  e.ncp = w.ncp;
  e.bound2 = (float)(1.0 + 1e-6);
  e.status = p->d_status;
  // the first step's slices, at the scales of the states' own maxima
  if (nsteps > 0) {
    k_band_rowmax<<<nc, 256, 0, s>>>(w.x[0], n, w.npl, w.kmax[1]);
    k_band_slice<<<dim3(w.ncp / 64, w.npl / 16), 256, 0, s>>>(w.x[0], n, w.npl, nc, w.npl, w.ncp, w.astride,
                                                              w.left[0], w.es[0], w.kmax[1]);
  }
  // step m's band (its gauge tables, its buffer of the pair)
  auto rows_of = [&](int m) {
    BandRows r{};
    r.cf = w.cf + (size_t)m * w.nrows;
    r.rot = w.rot + (size_t)m * w.nrows;
    r.right = w.right[m & 1];
    r.et = w.et[m & 1];
    r.rstride = w.rstride;
    r.ph_re = p->phase_re;
    r.ph_im = p->phase_im;
    r.n = n;
    r.nrows = w.nrows;
    r.L = L;
    r.kh = w.kh;
    return r;
  };
  const bool fold = w.ncp >= BAND_FORM_MIN_STATES;  // the next band formed inside each product
  int cur = 0;
  for (int m = 0; m < nsteps; ++m) {
    const int b = m & 1, nb = b ^ 1;
    if (m == 0 || !fold) k_band_rows<<<w.nrows / BAND_ROWS_PER_CTA, 32 * BAND_ROWS_PER_CTA, 0, s>>>(rows_of(m), coef);
    // X_m = P_m X_{m-1}, X_m's slices for the next step at the scales X_{m-1}'s maxima predict,
    // and P_{m+1} formed alongside when folded (into the other band buffer, which product m-1 read)
    e.et = w.et[b];
    e.out = w.x[cur ^ 1];
    e.kmax = w.kmax[b];
    e.es = w.es[b];
    e.lnext = w.left[nb];
    e.kprev = w.kmax[nb];
    e.write_states = m == nsteps - 1;
    fq_ktimer_start(p, s, "k_oz_band");
    const int form = fold && m + 1 < nsteps;
    k_oz_band<<<std::min(ntiles, sms), BAND_THREADS, BAND_SMEM, s>>>(maps[b], tiles_j, tiles_i, w.npl, w.kh, e,
                                                                     rows_of(form ? m + 1 : m), coef, form);
    fq_ktimer_stop(p, s);
    // the slice scales of X_m, and the states that outgrew their predicted scale cut again
    k_band_fixup<<<w.ncp / 8, 256, 0, s>>>(w.x[cur ^ 1], n, w.npl, nc, w.npl, w.ncp, w.astride, w.left[nb],
                                           w.es[nb], w.kmax[nb], w.kmax[b], w.ovf);
    cur ^= 1;
  }
  if (transpose_out) {
    dim3 g((n + 31) / 32, (n + 31) / 32), b(32, 8);
    k_band_store_t<<<g, b, 0, s>>>(w.x[cur], (double2*)x, n, w.npl);
  } else {
    k_band_store<<<band_grid((size_t)nc * n), 256, 0, s>>>(w.x[cur], (double2*)x, nc, n, w.npl);
  }
  cudaError_t e2 = cudaGetLastError();
  if (e2 != cudaSuccess) return fq_cuda_fail(e2, "band chain");
  return FQ_OK;
}
