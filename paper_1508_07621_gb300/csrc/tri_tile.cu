// Tiled tridiagonal chain (FP64 or FP32): one launch per step; each CTA carries one segment of one
// state through all L products of the step on chip and writes it back, so HBM sees the state
// once per step instead of five times per product.
//
// The step works in the real gauge frame of Omega~_m (gauge.cuh): X_m = D_m P(Omega'_m) D_m^+
// X_{m-1} with P(x) = e^{-i beta h} sum_k c_k T_k(x), c_k = (-i)^k a_k (Eqs. 10 and 12), applied by
// Clenshaw's backward recurrence.  A CTA holds NT * EPT consecutive rows: its segment of
// seg = NT * EPT - 2L rows plus L halo rows on each side.  Every product can be wrong only one
// row further in from the tile's edge (the rows beyond it are taken as zero), so after the L
// products of a step the segment's rows are exact; only those are written.
//
// FQ_DF32 runs the same step in double-float arithmetic: every value is an unevaluated sum
// hi + lo of two FP32 numbers (Dekker's splitting, Knuth's two-sum, and two-product by FMA), so
// the products keep about 48 significant bits on the FP32 pipes, which GB300 runs at many times
// its FP64 rate.  States stay FP64 in HBM between steps.
//
// Layout: states as rows, planar re / im planes [nc][ld] (the streaming kernel's layout).
// Per step and row: (2 d, 2 e') and (cos theta, sin theta) of D_m, in the kernel's precision,
// computed once per call in FP64 by k_gauge_tile.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "dfl.cuh"
#include "gauge.cuh"
#include "internal.h"

namespace {

constexpr int TILE_NT = 256;
constexpr int TILE_EPT = 8;
constexpr int TILE_ROWS = TILE_NT * TILE_EPT;
constexpr int TILE_MAXL = 128;

template <typename T>
struct TileCoef {
  T c[TILE_MAXL + 1];  // |c_k|: c_k = c[k] for even k (real, sign included), i c[k] for odd k
};

template <typename T>
struct Tile {
  using T2 = typename V2<T>::t;
  static constexpr int NW = TILE_NT / 32;
  T2* slot_last;   // [2][NW]
  T2* slot_first;  // [2][NW]
  int lane, warp;

  // rows i0 - 1 and i0 + EPT of x (neighbouring threads; zero beyond the tile)
  __device__ __forceinline__ void halo(const T2 (&x)[TILE_EPT], int par, T2& left, T2& right) {
    T lr = __shfl_up_sync(0xffffffffu, x[TILE_EPT - 1].x, 1);
    T li = __shfl_up_sync(0xffffffffu, x[TILE_EPT - 1].y, 1);
    T rr = __shfl_down_sync(0xffffffffu, x[0].x, 1);
    T ri = __shfl_down_sync(0xffffffffu, x[0].y, 1);
    if (lane == 31) slot_last[par * NW + warp] = x[TILE_EPT - 1];
    if (lane == 0) slot_first[par * NW + warp] = x[0];
    __syncthreads();
    if (lane == 0) {
      const T2 w = warp > 0 ? slot_last[par * NW + warp - 1] : T2{0, 0};
      lr = w.x;
      li = w.y;
    }
    if (lane == 31) {
      const T2 w = warp < NW - 1 ? slot_first[par * NW + warp + 1] : T2{0, 0};
      rr = w.x;
      ri = w.y;
    }
    left = T2{lr, li};
    right = T2{rr, ri};
  }

  // out = c v + (2 Omega' x) - out (HALF: c v + Omega' x - out, the closing sum), c = cc (real) or
  // i cc (IM): four FMAs per component, five for the closing sum
  template <bool IM, bool HALF>
  __device__ __forceinline__ void apply(const T2 (&x)[TILE_EPT], T2 (&out)[TILE_EPT], const T2 (&v)[TILE_EPT],
                                        const T (&d)[TILE_EPT], const T (&e)[TILE_EPT], T el0, T cc, int par) {
    T2 left, right;
    halo(x, par, left, right);
#pragma unroll
    for (int q = 0; q < TILE_EPT; ++q) {
      const T2 xm = q == 0 ? left : x[q - 1];
      const T2 xp = q == TILE_EPT - 1 ? right : x[q + 1];
      const T el = q == 0 ? el0 : e[q - 1];
      T ar, ai;
      if (HALF) {
        ar = fma((T)0.5, fma(d[q], x[q].x, fma(el, xm.x, e[q] * xp.x)), -out[q].x);
        ai = fma((T)0.5, fma(d[q], x[q].y, fma(el, xm.y, e[q] * xp.y)), -out[q].y);
      } else {
        ar = fma(d[q], x[q].x, fma(el, xm.x, fma(e[q], xp.x, -out[q].x)));
        ai = fma(d[q], x[q].y, fma(el, xm.y, fma(e[q], xp.y, -out[q].y)));
      }
      if (IM) {
        out[q] = T2{fma(-cc, v[q].y, ar), fma(cc, v[q].x, ai)};
      } else {
        out[q] = T2{fma(cc, v[q].x, ar), fma(cc, v[q].y, ai)};
      }
    }
  }
};

template <typename T>
__global__ void __launch_bounds__(TILE_NT)
k_tri_tile(const typename V2<T>::t* __restrict__ cf, const typename V2<T>::t* __restrict__ rot,
           const T* __restrict__ xr, const T* __restrict__ xi, T* __restrict__ yr, T* __restrict__ yi, int n, int ld,
           int L, int seg, TileCoef<T> coef, T ph_re, T ph_im, T bound2, unsigned int* status) {
  using T2 = typename V2<T>::t;
  __shared__ T2 slots[4 * Tile<T>::NW];
  Tile<T> tl;
  tl.slot_last = slots;
  tl.slot_first = slots + 2 * Tile<T>::NW;
  tl.lane = threadIdx.x & 31;
  tl.warp = threadIdx.x >> 5;
  const size_t j = blockIdx.y;
  const int first = blockIdx.x * seg;   // first row this CTA writes
  const int i0 = first - L + (int)threadIdx.x * TILE_EPT;
  T2 v[TILE_EPT], A[TILE_EPT], B[TILE_EPT];
  T d[TILE_EPT], e[TILE_EPT];
#pragma unroll
  for (int q = 0; q < TILE_EPT; ++q) {
    const int i = i0 + q;
    if (i >= 0 && i < n) {
      const T x_r = xr[j * ld + i], x_i = xi[j * ld + i];
      const T2 r = rot[i], c = cf[i];
      v[q] = T2{r.x * x_r + r.y * x_i, r.x * x_i - r.y * x_r};  // D^+ x
      d[q] = c.x;
      e[q] = c.y;
    } else {
      v[q] = T2{0, 0};
      d[q] = 0;
      e[q] = 0;
    }
  }
  // e' of the row before this thread's first row (constant over the step)
  T el0 = __shfl_up_sync(0xffffffffu, e[TILE_EPT - 1], 1);
  if (tl.lane == 0) {
    el0 = 0;
    if (i0 > 0 && i0 - 1 < n) el0 = cf[i0 - 1].y;
  }
  // b_L = c_L v, b_{L+1} = 0
  const T cL = coef.c[L];
#pragma unroll
  for (int q = 0; q < TILE_EPT; ++q) {
    A[q] = (L & 1) ? T2{-cL * v[q].y, cL * v[q].x} : T2{cL * v[q].x, cL * v[q].y};
    B[q] = T2{0, 0};
  }
  int k = L - 1, par = 0;
  // b_k = c_k v + 2 Omega' b_{k+1} - b_{k+2}; two per iteration so the array roles stay static
  while (k >= 2) {
    if (k & 1) tl.template apply<true, false>(A, B, v, d, e, el0, coef.c[k], par);
    else tl.template apply<false, false>(A, B, v, d, e, el0, coef.c[k], par);
    par ^= 1;
    --k;
    if (k & 1) tl.template apply<true, false>(B, A, v, d, e, el0, coef.c[k], par);
    else tl.template apply<false, false>(B, A, v, d, e, el0, coef.c[k], par);
    par ^= 1;
    --k;
  }
  if (k == 1) {  // b_1 into B, then sum = c_0 v + Omega' b_1 - b_2 into A
    tl.template apply<true, false>(A, B, v, d, e, el0, coef.c[1], par);
    par ^= 1;
    tl.template apply<false, true>(B, A, v, d, e, el0, coef.c[0], par);
  } else {  // b_1 in A, b_2 in B: sum into B, then moved to A
    tl.template apply<false, true>(A, B, v, d, e, el0, coef.c[0], par);
#pragma unroll
    for (int q = 0; q < TILE_EPT; ++q) A[q] = B[q];
  }
  // X = D e^{-i beta h} sum on this CTA's own rows
  bool bad = false;
#pragma unroll
  for (int q = 0; q < TILE_EPT; ++q) {
    const int i = i0 + q;
    if (i >= first && i < first + seg && i < n) {
      const T2 y = T2{ph_re * A[q].x - ph_im * A[q].y, ph_re * A[q].y + ph_im * A[q].x};
      const T2 r = rot[i];
      const T o_r = r.x * y.x - r.y * y.y, o_i = r.x * y.y + r.y * y.x;
      bad |= !(o_r * o_r + o_i * o_i <= bound2);
      yr[j * ld + i] = o_r;
      yi[j * ld + i] = o_i;
    }
  }
  if (bad) atomicOr(status, FQ_BIT_BOUND);
}

// ---------------------------------------------------------------------------- double-float
// 4 rows a thread and an 80-register cap (a few spills) let three CTAs (24 warps) share an SM:
// the double-float FMA chains are long, and latency, not the FP32 pipe, limits fewer warps.
constexpr int DFL_NT = 256;
constexpr int DFL_EPT = 4;
constexpr int DFL_ROWS = DFL_NT * DFL_EPT;
struct DflTile {
  static constexpr int NW = DFL_NT / 32;
  dflc* slot_last;   // [2][NW]
  dflc* slot_first;  // [2][NW]
  int lane, warp;

  __device__ __forceinline__ static dflc shfl(dflc a, bool up) {
    dflc r;
    if (up) {
      r.h.x = __shfl_up_sync(0xffffffffu, a.h.x, 1);
      r.h.y = __shfl_up_sync(0xffffffffu, a.h.y, 1);
      r.l.x = __shfl_up_sync(0xffffffffu, a.l.x, 1);
      r.l.y = __shfl_up_sync(0xffffffffu, a.l.y, 1);
    } else {
      r.h.x = __shfl_down_sync(0xffffffffu, a.h.x, 1);
      r.h.y = __shfl_down_sync(0xffffffffu, a.h.y, 1);
      r.l.x = __shfl_down_sync(0xffffffffu, a.l.x, 1);
      r.l.y = __shfl_down_sync(0xffffffffu, a.l.y, 1);
    }
    return r;
  }

  __device__ __forceinline__ void halo(const dflc (&x)[DFL_EPT], int par, dflc& left, dflc& right) {
    dflc l = shfl(x[DFL_EPT - 1], true);
    dflc r = shfl(x[0], false);
    if (lane == 31) slot_last[par * NW + warp] = x[DFL_EPT - 1];
    if (lane == 0) slot_first[par * NW + warp] = x[0];
    __syncthreads();
    const dflc z = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    if (lane == 0) l = warp > 0 ? slot_last[par * NW + warp - 1] : z;
    if (lane == 31) r = warp < NW - 1 ? slot_first[par * NW + warp + 1] : z;
    left = l;
    right = r;
  }

  // out = c v + (2 Omega' x) - out, or with Omega' x (HALF); c = cc or i cc (IM); all double-float
  template <bool IM, bool HALF>
  __device__ __forceinline__ void apply(const dflc (&x)[DFL_EPT], dflc (&out)[DFL_EPT], const dflc (&v)[DFL_EPT],
                                        const dfl (&d)[DFL_EPT], const dfl (&e)[DFL_EPT], dfl el0, dfl cc, int par) {
    dflc left, right;
    halo(x, par, left, right);
#pragma unroll
    for (int q = 0; q < DFL_EPT; ++q) {
      const dflc xm = q == 0 ? left : x[q - 1];
      const dflc xp = q == DFL_EPT - 1 ? right : x[q + 1];
      dfl dq = d[q], el = q == 0 ? el0 : e[q - 1], eh = e[q];
      if (HALF) {  // the closing sum uses Omega' = (stored operator) / 2, halved exactly
        dq = {0.5f * dq.h, 0.5f * dq.l};
        el = {0.5f * el.h, 0.5f * el.l};
        eh = {0.5f * eh.h, 0.5f * eh.l};
      }
      const dflc acc = dflc_fma(dq, x[q], dflc_fma(el, xm, dflc_fma(eh, xp, dflc_neg(out[q]))));
      out[q] = IM ? dflc_ifma(cc, v[q], acc) : dflc_fma(cc, v[q], acc);
    }
  }
};

struct DflCoef {
  dfl c[TILE_MAXL + 1];  // as TileCoef: c_k = c[k] (even k) or i c[k] (odd k)
};

// One step of the double-float tiled chain; states FP64 planar in HBM.
__global__ void __launch_bounds__(DFL_NT, 3)
k_tri_tile_dfl(const dfl2* __restrict__ cf, const dfl2* __restrict__ rot, const double* __restrict__ xr,
               const double* __restrict__ xi, double* __restrict__ yr, double* __restrict__ yi, int n, int ld, int L,
               int seg, DflCoef coef, double ph_re, double ph_im, double bound2, unsigned int* status) {
  __shared__ dflc slots[4 * DflTile::NW];
  DflTile tl;
  tl.slot_last = slots;
  tl.slot_first = slots + 2 * DflTile::NW;
  tl.lane = threadIdx.x & 31;
  tl.warp = threadIdx.x >> 5;
  const size_t j = blockIdx.y;
  const int first = blockIdx.x * seg;
  const int i0 = first - L + (int)threadIdx.x * DFL_EPT;
  const dfl zero = {0.f, 0.f};
  const dflc zc = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  dflc v[DFL_EPT], A[DFL_EPT], B[DFL_EPT];
  dfl d[DFL_EPT], e[DFL_EPT];
#pragma unroll
  for (int q = 0; q < DFL_EPT; ++q) {
    const int i = i0 + q;
    if (i >= 0 && i < n) {
      const double x_r = xr[j * ld + i], x_i = xi[j * ld + i];
      const dfl2 r = rot[i], c = cf[i];
      const double rc = dfl_value(r.x), rs = dfl_value(r.y);
      const dfl vr = dfl_of(rc * x_r + rs * x_i), vi = dfl_of(rc * x_i - rs * x_r);  // D^+ x in FP64
      v[q] = {make_float2(vr.h, vi.h), make_float2(vr.l, vi.l)};
      d[q] = c.x;
      e[q] = c.y;
    } else {
      v[q] = zc;
      d[q] = zero;
      e[q] = zero;
    }
  }
  dfl el0;
  el0.h = __shfl_up_sync(0xffffffffu, e[DFL_EPT - 1].h, 1);
  el0.l = __shfl_up_sync(0xffffffffu, e[DFL_EPT - 1].l, 1);
  if (tl.lane == 0) {
    el0 = zero;
    if (i0 > 0 && i0 - 1 < n) el0 = cf[i0 - 1].y;
  }
  // b_L = c_L v (L odd: i cL v)
  const dfl cL = coef.c[L];
#pragma unroll
  for (int q = 0; q < DFL_EPT; ++q) {
    A[q] = (L & 1) ? dflc_ifma(cL, v[q], zc) : dflc_fma(cL, v[q], zc);
    B[q] = zc;
  }
  int k = L - 1, par = 0;
  while (k >= 2) {
    if (k & 1) tl.apply<true, false>(A, B, v, d, e, el0, coef.c[k], par);
    else tl.apply<false, false>(A, B, v, d, e, el0, coef.c[k], par);
    par ^= 1;
    --k;
    if (k & 1) tl.apply<true, false>(B, A, v, d, e, el0, coef.c[k], par);
    else tl.apply<false, false>(B, A, v, d, e, el0, coef.c[k], par);
    par ^= 1;
    --k;
  }
  if (k == 1) {
    tl.apply<true, false>(A, B, v, d, e, el0, coef.c[1], par);
    par ^= 1;
    tl.apply<false, true>(B, A, v, d, e, el0, coef.c[0], par);
  } else {
    tl.apply<false, true>(A, B, v, d, e, el0, coef.c[0], par);
#pragma unroll
    for (int q = 0; q < DFL_EPT; ++q) A[q] = B[q];
  }
  bool bad = false;
#pragma unroll
  for (int q = 0; q < DFL_EPT; ++q) {
    const int i = i0 + q;
    if (i >= first && i < first + seg && i < n) {
      const double sr = (double)A[q].h.x + (double)A[q].l.x, si = (double)A[q].h.y + (double)A[q].l.y;
      const double y_r = ph_re * sr - ph_im * si, y_i = ph_re * si + ph_im * sr;
      const dfl2 r = rot[i];
      const double rc = dfl_value(r.x), rs = dfl_value(r.y);
      const double o_r = rc * y_r - rs * y_i, o_i = rc * y_i + rs * y_r;
      bad |= !(o_r * o_r + o_i * o_i <= bound2);
      yr[j * ld + i] = o_r;
      yi[j * ld + i] = o_i;
    }
  }
  if (bad) atomicOr(status, FQ_BIT_BOUND);
}

fq_status dfl_chain(fq_plan* p, const double* x0, double* x, int nc, int m_begin, int m_end, int identity,
                    int transpose_out, void* ws, cudaStream_t s) {
  const int n = p->n, ld = (n + 3) & ~3, nsteps = m_end - m_begin, L = p->L;
  const int seg = DFL_ROWS - 2 * L;
  dfl2* cf = (dfl2*)ws;
  dfl2* rot = cf + (size_t)nsteps * ld;
  double* bufs = (double*)(rot + (size_t)nsteps * ld);
  const size_t plane = (size_t)nc * ld;
  fq_blk<double> b[2] = {{bufs, bufs + plane}, {bufs + 2 * plane, bufs + 3 * plane}};
  GaugeArgs ga{p->n, p->steps, p->d_h0, p->d_h0o, p->d_h1, p->d_k, p->d_scal, p->sbeta};
  k_gauge_tile<dfl><<<nsteps, GAUGE_NT, 0, s>>>(ga, ld, m_begin, cf, rot);
  if (identity) fq_launch_identity_f64(b[0], nc, n, ld, s);
  else fq_launch_load_states(x0, b[0], nc, n, ld, s);
  DflCoef coef{};
  for (int k = 0; k <= L; ++k) {
    const double a = p->cheb[k];
    const double c = (k & 3) == 0 || (k & 3) == 3 ? a : -a;
    const float h = (float)c;
    coef.c[k] = {h, (float)(c - (double)h)};
  }
  const int segs = (n + seg - 1) / seg;
  int cur = 0;
  for (int m = 0; m < nsteps; ++m) {
    for (int r0 = 0; r0 < nc; r0 += 65535) {
      const int rows = nc - r0 < 65535 ? nc - r0 : 65535;
      const size_t o = (size_t)r0 * ld;
      fq_ktimer_start(p, s, "k_tri_tile_dfl");
      k_tri_tile_dfl<<<dim3(segs, rows), DFL_NT, 0, s>>>(cf + (size_t)m * ld, rot + (size_t)m * ld, b[cur].re + o,
                                                          b[cur].im + o, b[cur ^ 1].re + o, b[cur ^ 1].im + o, n, ld,
                                                          L, seg, coef, p->phase_re, p->phase_im, 1.0 + 1e-9,
                                                          p->d_status);
      fq_ktimer_stop(p, s);
    }
    cur ^= 1;
  }
  if (transpose_out) fq_launch_store_transpose_f64(b[cur], x, n, ld, s);
  else fq_launch_store_states_f64(b[cur], x, nc, n, ld, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fq_cuda_fail(e, "double-float tiled chain");
  return FQ_OK;
}

// state load / store helpers of the streaming path, by precision
void load_block(const double* x0, fq_blk<double> b, int nc, int n, int ld, cudaStream_t s) {
  fq_launch_load_states(x0, b, nc, n, ld, s);
}
void load_block(const double* x0, fq_blk<float> b, int nc, int n, int ld, cudaStream_t s) {
  fq_launch_load_states_f32(x0, b, nc, n, ld, s);
}
void identity_block(fq_blk<double> b, int nc, int n, int ld, cudaStream_t s) { fq_launch_identity_f64(b, nc, n, ld, s); }
void identity_block(fq_blk<float> b, int nc, int n, int ld, cudaStream_t s) { fq_launch_identity_f32(b, nc, n, ld, s); }
void store_block(fq_blk<double> b, double* x, int nc, int n, int ld, bool transpose, cudaStream_t s) {
  if (transpose) fq_launch_store_transpose_f64(b, x, n, ld, s);
  else fq_launch_store_states_f64(b, x, nc, n, ld, s);
}
void store_block(fq_blk<float> b, double* x, int nc, int n, int ld, bool transpose, cudaStream_t s) {
  if (transpose) fq_launch_store_transpose_f32(b, x, n, ld, s);
  else fq_launch_store_states_f32(b, x, nc, n, ld, s);
}

template <typename T>
TileCoef<T> tile_coef(const fq_plan* p) {
  TileCoef<T> c{};
  for (int k = 0; k <= p->L; ++k) {
    // c_k = (-i)^k a_k: k % 4 = 0: a, 1: -i a, 2: -a, 3: i a; odd k are stored as the factor of i
    const double a = p->cheb[k];
    c.c[k] = (T)((k & 3) == 0 || (k & 3) == 3 ? a : -a);
  }
  return c;
}

template <typename T>
fq_status tile_chain(fq_plan* p, const double* x0, double* x, int nc, int m_begin, int m_end, int identity,
                     int transpose_out, void* ws, cudaStream_t s) {
  using T2 = typename V2<T>::t;
  const int n = p->n, ld = (n + 3) & ~3, nsteps = m_end - m_begin, L = p->L;
  const int seg = TILE_ROWS - 2 * L;
  T2* cf = (T2*)ws;
  T2* rot = cf + (size_t)nsteps * ld;
  T* bufs = (T*)(rot + (size_t)nsteps * ld);
  const size_t plane = (size_t)nc * ld;
  fq_blk<T> b[2] = {{bufs, bufs + plane}, {bufs + 2 * plane, bufs + 3 * plane}};
  GaugeArgs ga{p->n, p->steps, p->d_h0, p->d_h0o, p->d_h1, p->d_k, p->d_scal, p->sbeta};
  k_gauge_tile<T><<<nsteps, GAUGE_NT, 0, s>>>(ga, ld, m_begin, cf, rot);
  if (identity) identity_block(b[0], nc, n, ld, s);
  else load_block(x0, b[0], nc, n, ld, s);
  const TileCoef<T> coef = tile_coef<T>(p);
  const T b2 = (T)(1.0 + (sizeof(T) == 8 ? 1e-9 : 2e-3));
  const int segs = (n + seg - 1) / seg;
  int cur = 0;
  for (int m = 0; m < nsteps; ++m) {
    for (int r0 = 0; r0 < nc; r0 += 65535) {  // gridDim.y limit
      const int rows = nc - r0 < 65535 ? nc - r0 : 65535;
      const size_t o = (size_t)r0 * ld;
      k_tri_tile<T><<<dim3(segs, rows), TILE_NT, 0, s>>>(cf + (size_t)m * ld, rot + (size_t)m * ld,
                                                         b[cur].re + o, b[cur].im + o, b[cur ^ 1].re + o,
                                                         b[cur ^ 1].im + o, n, ld, L, seg, coef, (T)p->phase_re,
                                                         (T)p->phase_im, b2, p->d_status);
    }
    cur ^= 1;
  }
  store_block(b[cur], x, nc, n, ld, transpose_out != 0, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fq_cuda_fail(e, "tiled tridiagonal chain");
  return FQ_OK;
}

}  // namespace

int fq_tile_supported(int L) { return L >= 1 && L <= TILE_MAXL && 2 * L < TILE_ROWS / 2; }

size_t fq_tile_workspace(const fq_plan* p, int nc, int nsteps) {
  const size_t ld = (p->n + 3) & ~3;
  if (p->precision == FQ_DF32)  // double-float coefficients (16 B a pair), FP64 states
    return 2 * (size_t)nsteps * ld * sizeof(dfl2) + 4 * (size_t)nc * ld * sizeof(double);
  const size_t es = p->precision == FQ_FP64 ? sizeof(double) : sizeof(float);
  return 2 * (size_t)nsteps * ld * 2 * es + 4 * (size_t)nc * ld * es;
}

fq_status fq_tile_propagate(fq_plan* p, const double* x0, double* x, int nc, int m_begin, int m_end, int identity,
                            int transpose_out, void* ws, cudaStream_t s) {
  if (p->precision == FQ_FP64)
    return tile_chain<double>(p, x0, x, nc, m_begin, m_end, identity, transpose_out, ws, s);
  if (p->precision == FQ_DF32) return dfl_chain(p, x0, x, nc, m_begin, m_end, identity, transpose_out, ws, s);
  return tile_chain<float>(p, x0, x, nc, m_begin, m_end, identity, transpose_out, ws, s);
}
