// Resident tridiagonal chain (FP32): one CTA carries one state through all steps
// m_begin..m_end-1 without touching HBM in between.
//
// Gauge: Omega~_m is Hermitian tridiagonal with complex off-diagonal e_k.  With
// D_m = diag(e^{i theta_k}), theta_{k+1} - theta_k = phi_k = arg(e_k) reduced to (-pi/2, pi/2],
// Omega~_m = D_m Omega'_m D_m^+ where Omega'_m is REAL symmetric tridiagonal (off-diagonal
// e'_k = +-|e_k|).  Hence exp(-i Omega_m) = e^{-i beta h} D_m P(Omega'_m) D_m^+ and the chain
// runs in the frame of each step: v <- (D_m^+ D_{m-1}) v before step m, X = D_last v at the end.
// A real operator acts on the (re, im) pair of every entry alike, so each product is four
// packed FP32x2 FMAs per entry (c v - b_{k+2}, then the three operator entries).
//
// Each step applies sum_{k=0}^{L} c_k T_k(Omega') v with c_k = (-i)^k a_k (Eqs. 10 and 12:
// psi_k = (-i)^k T_k(Omega~) v) by Clenshaw's backward recurrence
//     b_{L+1} = b_{L+2} = 0,  b_k = c_k v + 2 Omega' b_{k+1} - b_{k+2}  (k = L..1),
//     sum = c_0 v + Omega' b_1 - b_2,
// which needs the same L products as the forward recurrence of Eq. 10 but only two live
// vectors besides v.  Then X_m = e^{-i beta h} sum.
//
// Layout: NT threads (256 x 40 rows above 9216 rows, 512 x <= 18 below, 256 x 2 or 4 up to 1024);
// thread t owns rows i = t*EPT .. t*EPT+EPT-1 (EPT even).  b_{k+1}, b_{k+2} live in registers as
// (re, im) pairs; v and the step's (2 d, 2 e') pairs live in shared memory as float4 holding rows
// (2p, 2p+1) of thread t at [p][t], so one conflict-free 16-byte access serves two rows.  The
// per-step coefficient and rotation arrays are written in global memory in exactly that order
// ("resident order"), so their loads are coalesced.  Each sweep over a thread's rows applies two
// products (Chain::pass); the two-row halo of b_{k+1} crosses lanes by warp shuffles and warps
// through small double-buffered shared arrays (one __syncthreads per two products).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "gauge.cuh"
#include "internal.h"

namespace {

constexpr int RES_MAXNW = 32;
constexpr int RES_MAXL = 128;
struct ResCoef {
  float cr[RES_MAXL + 1];  // c_k = (-i)^k a_k: real for even k, imaginary for odd k
  float ci[RES_MAXL + 1];
};

struct ResShared {
  float4 slot_last[2][RES_MAXNW];  // last two rows of each warp's lane 31
  float red[RES_MAXNW];
  float tot;           // squared norm of the initial state
  float lim_state;     // bound on |X_m entry|^2
  float lim_clenshaw;  // bound on |b_1 entry|^2
  unsigned int bad;    // set by any thread whose check failed
};

// Position of row i in resident order (float2 units) for NT threads of EPT rows each.
__host__ __device__ __forceinline__ size_t res_index(int i, int nt, int ept) {
  const int t = i / ept, q = i - t * ept;
  return ((size_t)(q >> 1) * nt + t) * 2 + (q & 1);
}

// CTA s < nsteps (step m = m_begin + s): cf[s][k] = (2 d_k, 2 e'_k) and
//   rot[s][k] = e^{i (theta^{m-1}_k - theta^m_k)}  (theta^{m_begin - 1} := 0: input frame);
// CTA s = nsteps: rot[nsteps][k] = e^{i theta^{m_end - 1}_k} (back to the original frame).
// FP64 arithmetic throughout (the Magnus combination and rescaling stay FP64), FP32 stores.
__global__ void __launch_bounds__(GAUGE_NT) k_gauge_coeffs(GaugeArgs p, int ld, int m_begin, int nsteps, int rnt,
                                                           int rept, float2* __restrict__ cf, float2* __restrict__ rot) {
  const size_t stride = (size_t)rnt * rept;  // one step, resident order; rows >= ld stay as set below
  __shared__ double sw[64];
  const int s = blockIdx.x;
  const int C = (ld + GAUGE_NT - 1) / GAUGE_NT;
  const int k0 = threadIdx.x * C;
  double thA[GAUGE_MAXC], thB[GAUGE_MAXC];
  if (s < nsteps) {
    const int m = m_begin + s;
    phases(p, m, ld, C, thA, sw);
    phases(p, s == 0 ? -1 : m - 1, ld, C, thB, sw);
#pragma unroll
    for (int q = 0; q < GAUGE_MAXC; ++q) {
      const int k = k0 + q;
      if (q < C && k < ld) {
        const double d = k < p.n ? p.scal[m] * p.h0d[k] + p.scal[p.M + m] * p.h1d[k] - p.sbeta : 0.0;
        double er, ei;
        offdiag(p, m, k, er, ei);
        double sp, cp;
        sincos(reduced_arg(er, ei), &sp, &cp);
        const double ep = er * cp + ei * sp;  // e_k e^{-i phi_k}, whose imaginary part is 0
        cf[s * stride + res_index(k, rnt, rept)] = make_float2((float)(2.0 * d), (float)(2.0 * ep));
        double sr, cr;
        sincos(thB[q] - thA[q], &sr, &cr);
        rot[s * stride + res_index(k, rnt, rept)] = make_float2((float)cr, (float)sr);
      }
    }
  } else {
    phases(p, m_begin + nsteps - 1, ld, C, thA, sw);
#pragma unroll
    for (int q = 0; q < GAUGE_MAXC; ++q) {
      const int k = k0 + q;
      if (q < C && k < ld) {
        double sr, cr;
        sincos(thA[q], &sr, &cr);
        rot[s * stride + res_index(k, rnt, rept)] = make_float2((float)cr, (float)sr);
      }
    }
  }
}

// ---------------------------------------------------------------------------- chain
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 lo2(float4 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ float2 hi2(float4 a) { return make_float2(a.z, a.w); }

// c v for a real c (IM = false) or an imaginary c = i cc (IM = true)
template <bool IM>
__device__ __forceinline__ float2 cvec(float cc, float2 vv) {
  return IM ? f2(-cc * vv.y, cc * vv.x) : f2(cc * vv.x, cc * vv.y);
}

// one row of a Clenshaw product: c v - o + (2 Omega' x)_row, where the row of the stored operator
// 2 Omega' is (el, d, eh) on (xm, x0, xp).  Four packed FP32x2 FMAs for a real c.
template <bool IM>
__device__ __forceinline__ float2 row(float cc, float2 vv, float2 o, float d, float2 x0, float el, float2 xm, float eh,
                                      float2 xp) {
  float2 acc;
  if (IM) acc = f2(fmaf(-cc, vv.y, -o.x), fmaf(cc, vv.x, -o.y));
  else acc = __ffma2_rn(f2(cc, cc), vv, f2(-o.x, -o.y));
  acc = __ffma2_rn(f2(d, d), x0, acc);
  acc = __ffma2_rn(f2(el, el), xm, acc);
  return __ffma2_rn(f2(eh, eh), xp, acc);
}

// the closing product: c0 v - o + (1/2)(2 Omega' x)_row, c0 real
__device__ __forceinline__ float2 row_half(float cc, float2 vv, float2 o, float d, float2 x0, float el, float2 xm,
                                           float eh, float2 xp) {
  float2 s = __fmul2_rn(f2(d, d), x0);
  s = __ffma2_rn(f2(el, el), xm, s);
  s = __ffma2_rn(f2(eh, eh), xp, s);
  return __ffma2_rn(f2(0.5f, 0.5f), s, __ffma2_rn(f2(cc, cc), vv, f2(-o.x, -o.y)));
}

template <int NT, int EPT>
struct Chain {
  static constexpr int NW = NT / 32;
  static constexpr int NP = EPT / 2;
  const float4* v;   // [NP][NT] state in the step's frame, rows (2p, 2p+1)
  const float4* cf;  // [NP][NT] (2 d, 2 e') of rows (2p, 2p+1), e'_i = Omega'[i+1][i]
  float4* first2;    // [2][NT] first two rows of b_{k+1} per thread (exchange buffers)
  float4* bhalo;     // [NT] (b_k at row i0-1, b_k at row i0+EPT) per thread, carried between passes
  ResShared* sh;
  int t, lane, warp;

  // Publishes x's first two rows for the left neighbour (read back by right() after the sweep) and
  // returns rows i0-2, i0-1 (as (re, im, re, im)) of the left neighbour; zero before row 0.
  // One __syncthreads; the buffers alternate with par so that one barrier per pass suffices.
  __device__ __forceinline__ float4 exchange(const float2 (&x)[EPT], int par) {
    float4 l;
    l.x = __shfl_up_sync(0xffffffffu, x[EPT - 2].x, 1);
    l.y = __shfl_up_sync(0xffffffffu, x[EPT - 2].y, 1);
    l.z = __shfl_up_sync(0xffffffffu, x[EPT - 1].x, 1);
    l.w = __shfl_up_sync(0xffffffffu, x[EPT - 1].y, 1);
    if (lane == 31) sh->slot_last[par][warp] = make_float4(x[EPT - 2].x, x[EPT - 2].y, x[EPT - 1].x, x[EPT - 1].y);
    first2[par * NT + t] = make_float4(x[0].x, x[0].y, x[1].x, x[1].y);
    __syncthreads();
    if (lane == 0) l = warp > 0 ? sh->slot_last[par][warp - 1] : make_float4(0.f, 0.f, 0.f, 0.f);
    return l;
  }
  // rows i0+EPT, i0+EPT+1 as published by the right neighbour in exchange(); zero past the end
  __device__ __forceinline__ float4 right(int par) const {
    return t < NT - 1 ? first2[par * NT + t + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
  }

  // Two Clenshaw products in one sweep over the rows (Eqs. 10 and 12 in backward form):
  //   P1: b_k     = c_k v + 2 Omega' b_{k+1} - b_{k+2}   on rows i0-1 .. i0+EPT (own rows + one halo row a side)
  //   P2: b_{k-1} = c_{k-1} v + 2 Omega' b_k - b_{k+1}   on own rows (FINAL: the closing sum with Omega')
  // In: A = b_{k+1}, B = b_{k+2} (own rows), bhalo[t] = b_{k+2} on the halo rows (FIRST: all zero).
  // Out: A = b_{k-1}, B = b_k, bhalo[t] = b_k on the halo rows (only thread t touches bhalo[t]).  The operator and v rows of a pair are
  // read from shared memory once for both products; only b_{k+1} crosses threads (two rows a side).
  // K_ODD: c_k = i c1 and c_{k-1} = c2 real; otherwise c_k = c1 real and c_{k-1} = i c2.
  template <bool FIRST, bool FINAL, bool K_ODD>
  __device__ __forceinline__ void pass(float2 (&A)[EPT], float2 (&B)[EPT], float c1, float c2, int par) {
    constexpr bool IM1 = K_ODD, IM2 = !K_ODD;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float2 z2 = f2(0.f, 0.f);
    const float4 al = FIRST ? z4 : exchange(A, par);
    const float2 am2 = lo2(al), am1 = hi2(al);
    // row i0-1: (., 2e'_{i0-2}, 2d_{i0-1}, 2e'_{i0-1}) and its v
    const float4 cl = t > 0 ? cf[(NP - 1) * NT + t - 1] : z4;
    const float2 vl = t > 0 ? hi2(v[(NP - 1) * NT + t - 1]) : z2;
    const float2 nbl =
        FIRST ? cvec<IM1>(c1, vl) : row<IM1>(c1, vl, lo2(bhalo[t]), cl.z, am1, cl.y, am2, cl.w, A[0]);
    float4 cp = cl;  // operator of rows 2p-2, 2p-1
    float2 vp = vl;  // v of row 2p-1
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const int q = 2 * p;
      const float4 c = cf[p * NT + t];
      const float4 w = v[p * NT + t];
      float2 b0, b1;
      if (FIRST) {
        b0 = cvec<IM1>(c1, lo2(w));
        b1 = cvec<IM1>(c1, hi2(w));
      } else {
        b0 = row<IM1>(c1, lo2(w), B[q], c.x, A[q], cp.w, q == 0 ? am1 : A[q - 1], c.y, A[q + 1]);
        b1 = row<IM1>(c1, hi2(w), B[q + 1], c.z, A[q + 1], c.y, A[q], c.w,
                      q + 2 < EPT ? A[q + 2] : lo2(right(par)));
      }
      // P2 on row q-1 (its upper neighbour b0 is now known) and on row q
      if (p > 0) {
        const float2 o = FIRST ? z2 : A[q - 1];
        A[q - 1] = FINAL ? row_half(c2, vp, o, cp.z, B[q - 1], cp.y, q >= 2 ? B[q - 2] : nbl, cp.w, b0)
                         : row<IM2>(c2, vp, o, cp.z, B[q - 1], cp.y, q >= 2 ? B[q - 2] : nbl, cp.w, b0);
      }
      {
        const float2 o = FIRST ? z2 : A[q];
        A[q] = FINAL ? row_half(c2, lo2(w), o, c.x, b0, cp.w, q == 0 ? nbl : B[q - 1], c.y, b1)
                     : row<IM2>(c2, lo2(w), o, c.x, b0, cp.w, q == 0 ? nbl : B[q - 1], c.y, b1);
      }
      B[q] = b0;
      B[q + 1] = b1;
      cp = c;
      vp = hi2(w);
    }
    // row i0+EPT: (2d, 2e') of that row and its v
    const float2 cr = t < NT - 1 ? lo2(cf[t + 1]) : z2;
    const float2 vr = t < NT - 1 ? lo2(v[t + 1]) : z2;
    float2 nbr;
    if (FIRST) {
      nbr = cvec<IM1>(c1, vr);
    } else {
      const float4 ar = right(par);
      nbr = row<IM1>(c1, vr, hi2(bhalo[t]), cr.x, lo2(ar), cp.w, A[EPT - 1], cr.y, hi2(ar));
    }
    {
      const float2 o = FIRST ? z2 : A[EPT - 1];
      A[EPT - 1] = FINAL ? row_half(c2, vp, o, cp.z, B[EPT - 1], cp.y, B[EPT - 2], cp.w, nbr)
                         : row<IM2>(c2, vp, o, cp.z, B[EPT - 1], cp.y, B[EPT - 2], cp.w, nbr);
    }
    bhalo[t] = make_float4(nbl.x, nbl.y, nbr.x, nbr.y);
  }

  // The closing product alone (an even number L): B <- c0 v + Omega' A - B on own rows, A = b_1.
  __device__ __forceinline__ void single_final(const float2 (&A)[EPT], float2 (&B)[EPT], float c0, int par) {
    const float2 am1 = hi2(exchange(A, par));
    float el = t > 0 ? cf[(NP - 1) * NT + t - 1].w : 0.f;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const int q = 2 * p;
      const float4 c = cf[p * NT + t];
      const float4 w = v[p * NT + t];
      B[q] = row_half(c0, lo2(w), B[q], c.x, A[q], el, q == 0 ? am1 : A[q - 1], c.y, A[q + 1]);
      B[q + 1] =
          row_half(c0, hi2(w), B[q + 1], c.z, A[q + 1], c.y, A[q], c.w, q + 2 < EPT ? A[q + 2] : lo2(right(par)));
      el = c.w;
    }
  }

  // flags any entry of x with |x|^2 above lim
  __device__ __forceinline__ void check(const float2 (&x)[EPT], float lim) {
    bool ok = true;
#pragma unroll
    for (int q = 0; q < EPT; ++q) ok &= x[q].x * x[q].x + x[q].y * x[q].y <= lim;
    if (!ok) sh->bad = 1u;
  }

  // sum_{k=0}^{L} c_k T_k(Omega') v into A (c_k = (-i)^k a_k: imaginary exactly for odd k);
  // checks |b_1| against the Clenshaw bound.
  template <bool L_ODD>
  __device__ __forceinline__ void series(float2 (&A)[EPT], float2 (&B)[EPT], int L, const ResCoef& coef) {
    // c_k = i ci[k] for odd k, cr[k] for even k
    auto cc = [&](int k) { return (k & 1) ? coef.ci[k] : coef.cr[k]; };
    int par = 0;
    if (L_ODD && L == 1) {
      pass<true, true, true>(A, B, cc(1), cc(0), par);
      check(B, sh->lim_clenshaw);
      return;
    }
    pass<true, false, L_ODD>(A, B, cc(L), cc(L - 1), par);
    int k = L - 2;
    for (; k >= 2; k -= 2) {
      pass<false, false, L_ODD>(A, B, cc(k), cc(k - 1), par);
      par ^= 1;
    }
    if (L_ODD) {  // k == 1: the pair (1, 0) closes the series; B = b_1 afterwards
      pass<false, true, true>(A, B, cc(1), cc(0), par);
      check(B, sh->lim_clenshaw);
    } else {  // k == 0: A = b_1, B = b_2
      check(A, sh->lim_clenshaw);
      single_final(A, B, cc(0), par);
#pragma unroll
      for (int q = 0; q < EPT; ++q) A[q] = B[q];
    }
  }
};

template <int NT, int EPT>
__global__ void __launch_bounds__(NT, 1)
k_tri_resident(const float4* __restrict__ cf_all, const float4* __restrict__ rot_all, int n, int L, int nsteps,
               const double2* __restrict__ x0, double2* __restrict__ xout, int transpose_out, ResCoef coef,
               float ph_re, float ph_im, float clenshaw_bound, unsigned int* status) {
  using Ch = Chain<NT, EPT>;
  constexpr int NP = EPT / 2, NW = NT / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* sv = reinterpret_cast<float4*>(smem_raw);
  float4* scf = sv + NP * NT;
  Ch C;
  C.v = sv;
  C.cf = scf;
  C.first2 = sv + 2 * NP * NT;
  C.bhalo = sv + 2 * NP * NT + 2 * NT;
  C.sh = reinterpret_cast<ResShared*>(sv + 2 * NP * NT + 3 * NT);
  C.t = threadIdx.x;
  C.lane = threadIdx.x & 31;
  C.warp = threadIdx.x >> 5;
  const int t = threadIdx.x;
  const int j = blockIdx.x;  // state index
  const int i0 = t * EPT;
  const size_t stride = (size_t)NP * NT;  // one step of cf / rot, in float4

  // initial state (registers) and its squared norm (unitarity bounds every later entry by it)
  float2 A[EPT], B[EPT];
  float nrm = 0.f;
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const int i = i0 + q;
    float a = 0.f, b = 0.f;
    if (i < n) {
      if (x0) {
        const double2 zz = x0[(size_t)j * n + i];
        a = (float)zz.x;
        b = (float)zz.y;
      } else {
        a = i == j ? 1.f : 0.f;
      }
    }
    A[q] = f2(a, b);
    nrm = fmaf(a, a, fmaf(b, b, nrm));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
  if (C.lane == 0) C.sh->red[C.warp] = nrm;
  __syncthreads();
  if (t == 0) {
    float tot = 0.f;
    for (int w = 0; w < NW; ++w) tot += C.sh->red[w];
    C.sh->tot = tot;
    C.sh->lim_state = tot * 1.002f + 1e-30f;
    // |b_k| <= sum_j |c_j| |U_{j-k}(Omega')| |v| <= sum_j (j+1)|a_j| |v| while the spectrum of
    // Omega' lies in [-1, 1] (|U_n| <= n+1 there); outside it U_n grows exponentially.
    C.sh->lim_clenshaw = tot * clenshaw_bound * clenshaw_bound * 1.01f + 1e-30f;
    C.sh->bad = 0u;
  }

  for (int m = 0; m < nsteps; ++m) {
    const size_t off = (size_t)m * stride;
    // the next step's operator and rotation blocks into L2 while this step runs (one thread each)
    if (t < 2 && m + 1 < nsteps) {
      const float4* nxt = (t == 0 ? cf_all : rot_all) + off + stride;
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(nxt), "r"((unsigned)(stride * sizeof(float4)))
                   : "memory");
    }
    // every thread is done with the previous step's operator and state rows
    __syncthreads();
    // this step's (2 d, 2 e') and the frame change D_m^+ D_{m-1} of the state (coalesced)
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const int s = p * NT + t;
      const float4 c = cf_all[off + s];
      const float4 r = rot_all[off + s];
      scf[s] = c;
      const float2 a = A[2 * p], b = A[2 * p + 1];
      sv[s] = make_float4(r.x * a.x - r.y * a.y, r.x * a.y + r.y * a.x, r.z * b.x - r.w * b.y, r.z * b.y + r.w * b.x);
    }
    C.check(A, C.sh->lim_state);  // X_{m-1} (or the initial state)
    __syncthreads();
    if (L & 1) C.template series<true>(A, B, L, coef);
    else C.template series<false>(A, B, L, coef);
    // X_m = e^{-i beta h} sum (this step's frame)
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const float2 a = A[q];
      A[q] = f2(ph_re * a.x - ph_im * a.y, ph_re * a.y + ph_im * a.x);
    }
  }
  // back to the original frame: X = D_last v; unitarity check on the state's norm (a spectral
  // bound that is too tight keeps the entries small but makes the truncated series non-unitary)
  float nrm_end = 0.f;
  const size_t offr = (size_t)nsteps * stride;
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const float4 r = rot_all[offr + p * NT + t];
    const float2 a = A[2 * p], b = A[2 * p + 1];
    A[2 * p] = f2(r.x * a.x - r.y * a.y, r.x * a.y + r.y * a.x);
    A[2 * p + 1] = f2(r.z * b.x - r.w * b.y, r.z * b.y + r.w * b.x);
    nrm_end = fmaf(A[2 * p].x, A[2 * p].x, fmaf(A[2 * p].y, A[2 * p].y, nrm_end));
    nrm_end = fmaf(A[2 * p + 1].x, A[2 * p + 1].x, fmaf(A[2 * p + 1].y, A[2 * p + 1].y, nrm_end));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nrm_end += __shfl_xor_sync(0xffffffffu, nrm_end, o);
  __syncthreads();
  if (C.lane == 0) C.sh->red[C.warp] = nrm_end;
  __syncthreads();
  if (t == 0) {
    float tot_end = 0.f;
    for (int w = 0; w < NW; ++w) tot_end += C.sh->red[w];
    const float tot = C.sh->tot;
    if (!(fabsf(tot_end - tot) <= 1e-3f * tot + 1e-30f)) C.sh->bad = 1u;
  }
  __syncthreads();
  if (t == 0 && C.sh->bad) atomicOr(status, FQ_BIT_BOUND);
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const int i = i0 + q;
    if (i < n) {
      const double2 x = make_double2((double)A[q].x, (double)A[q].y);
      if (transpose_out) xout[(size_t)i * n + j] = x;
      else xout[(size_t)j * n + i] = x;
    }
  }
}

template <int NT, int EPT>
fq_status launch_cfg(const fq_plan* p, const float4* cf, const float4* rot, const double* x0, double* x,
                     int transpose_out, int nc, int nsteps, const ResCoef& coef, float bcl, cudaStream_t s) {
  const size_t smem = sizeof(float4) * (EPT + 3) * NT + sizeof(ResShared);
  static std::atomic<unsigned> attr_set{0};
  if (fq_first_on_device(attr_set)) {
    cudaError_t e =
        cudaFuncSetAttribute(k_tri_resident<NT, EPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return fq_cuda_fail(e, "resident kernel smem attribute");
  }
  fq_ktimer_start(p, s, "k_tri_resident");
  k_tri_resident<NT, EPT><<<nc, NT, smem, s>>>(cf, rot, p->n, p->L, nsteps, (const double2*)x0, (double2*)x,
                                                transpose_out, coef, (float)p->phase_re, (float)p->phase_im, bcl,
                                                p->d_status);
  fq_ktimer_stop(p, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fq_cuda_fail(e, "resident kernel launch");
  return FQ_OK;
}

// (threads, rows per thread) for dimension n; 0 threads if the resident kernel does not apply.
// Above 9216 rows, 256 x 40 (250 registers, no spills) beats 512 x 20, which has to fit in 128
// registers and spills; 1024 x 10 would have to fit in 64.
void res_config(int n, int* nt, int* ept) {
  *nt = 0;
  *ept = 0;
  if (n <= 256 * 4) {
    *nt = 256;
    *ept = n <= 512 ? 2 : 4;
    return;
  }
  const int need = (n + 511) / 512;
  if (need > 20) return;
  if (need > 18) {
    *nt = 256;
    *ept = 40;
    return;
  }
  *nt = 512;
  *ept = need + (need & 1);
}

}  // namespace

int fq_resident_supported(int n, int L) {
  int nt, ept;
  res_config(n, &nt, &ept);
  return nt > 0 && L <= RES_MAXL && L >= 1;
}

// (2 nsteps + 1) blocks of nt * ept float2 in resident order: the operator pairs of every step,
// then the frame rotation of every step plus the final one.
size_t fq_resident_coeff_bytes(int n, int steps) {
  int nt, ept;
  res_config(n, &nt, &ept);
  return (2 * (size_t)steps + 1) * (size_t)nt * ept * sizeof(float2);
}

void fq_launch_gauge_coeffs(const fq_plan* p, int m_begin, int nsteps, void* coeff, cudaStream_t s) {
  const int ld = (p->n + 3) & ~3;
  int nt, ept;
  res_config(p->n, &nt, &ept);
  float2* cf = (float2*)coeff;
  float2* rot = cf + (size_t)nsteps * nt * ept;
  // rows beyond ld (padding of the resident order) must hold cf = 0 and rot = 1: zero them
  // and let the kernel overwrite every row < ld; rot padding only multiplies zeros.
  cudaMemsetAsync(coeff, 0, fq_resident_coeff_bytes(p->n, nsteps), s);
  GaugeArgs ga{p->n, p->steps, p->d_h0, p->d_h0o, p->d_h1, p->d_k, p->d_scal, p->sbeta};
  k_gauge_coeffs<<<nsteps + 1, GAUGE_NT, 0, s>>>(ga, ld, m_begin, nsteps, nt, ept, cf, rot);
}

fq_status fq_launch_resident(const fq_plan* p, const void* coeff, const double* x0, double* x, int transpose_out,
                             int nc, int m_begin, int m_end, cudaStream_t s) {
  const int nsteps = m_end - m_begin;
  int nt, ept;
  res_config(p->n, &nt, &ept);
  const float4* cf = (const float4*)coeff;
  const float4* rot = cf + (size_t)nsteps * nt * ept / 2;
  ResCoef coef;
  double bcl = 0.0;
  for (int k = 0; k <= p->L; ++k) bcl += (k + 1) * fabs(p->cheb[k]);
  for (int k = 0; k <= p->L; ++k) {
    // (-i)^k a_k
    const double a = p->cheb[k];
    switch (k & 3) {
      case 0: coef.cr[k] = (float)a; coef.ci[k] = 0.f; break;
      case 1: coef.cr[k] = 0.f; coef.ci[k] = (float)-a; break;
      case 2: coef.cr[k] = (float)-a; coef.ci[k] = 0.f; break;
      default: coef.cr[k] = 0.f; coef.ci[k] = (float)a; break;
    }
  }
  const float b = (float)bcl;
  if (nt == 256 && ept == 2) return launch_cfg<256, 2>(p, cf, rot, x0, x, transpose_out, nc, nsteps, coef, b, s);
  if (nt == 256 && ept == 4) return launch_cfg<256, 4>(p, cf, rot, x0, x, transpose_out, nc, nsteps, coef, b, s);
  if (nt == 256 && ept == 40) return launch_cfg<256, 40>(p, cf, rot, x0, x, transpose_out, nc, nsteps, coef, b, s);
  switch (ept) {
    case 4: return launch_cfg<512, 4>(p, cf, rot, x0, x, transpose_out, nc, nsteps, coef, b, s);
    case 6: return launch_cfg<512, 6>(p, cf, rot, x0, x, transpose_out, nc, nsteps, coef, b, s);
    case 8: return launch_cfg<512, 8>(p, cf, rot, x0, x, transpose_out, nc, nsteps, coef, b, s);
    case 10: return launch_cfg<512, 10>(p, cf, rot, x0, x, transpose_out, nc, nsteps, coef, b, s);
    case 12: return launch_cfg<512, 12>(p, cf, rot, x0, x, transpose_out, nc, nsteps, coef, b, s);
    case 14: return launch_cfg<512, 14>(p, cf, rot, x0, x, transpose_out, nc, nsteps, coef, b, s);
    case 16: return launch_cfg<512, 16>(p, cf, rot, x0, x, transpose_out, nc, nsteps, coef, b, s);
    case 18: return launch_cfg<512, 18>(p, cf, rot, x0, x, transpose_out, nc, nsteps, coef, b, s);
    case 20: return launch_cfg<512, 20>(p, cf, rot, x0, x, transpose_out, nc, nsteps, coef, b, s);
    default: fq_set_error("resident kernel: n = %d too large", p->n); return FQ_EUNSUPPORTED;
  }
}
