// Resident tridiagonal chain (FP32): one CTA carries one state through all steps
// m_begin..m_end-1 without touching HBM in between.
//
// Gauge: Omega~_m is Hermitian tridiagonal with complex off-diagonal e_k.  With
// D_m = diag(e^{i theta_k}), theta_{k+1} - theta_k = phi_k = arg(e_k) reduced to (-pi/2, pi/2],
// Omega~_m = D_m Omega'_m D_m^+ where Omega'_m is REAL symmetric tridiagonal (off-diagonal
// e'_k = +-|e_k|).  Hence exp(-i Omega_m) = e^{-i beta h} D_m P(Omega'_m) D_m^+ and the chain
// runs in the frame of each step: v <- (D_m^+ D_{m-1}) v before step m, X = D_last v at the end.
// A real operator acts on the (re, im) pair of every entry alike, so each product is three
// packed FP32x2 FMAs per entry.
//
// Each step applies sum_{k=0}^{L} c_k T_k(Omega') v with c_k = (-i)^k a_k (Eqs. 10 and 12:
// psi_k = (-i)^k T_k(Omega~) v) by Clenshaw's backward recurrence
//     b_{L+1} = b_{L+2} = 0,  b_k = c_k v + 2 Omega' b_{k+1} - b_{k+2}  (k = L..1),
//     sum = c_0 v + Omega' b_1 - b_2,
// which needs the same L products as the forward recurrence of Eq. 10 but only two live
// vectors besides v.  Then X_m = e^{-i beta h} sum.
//
// Layout: NT threads (512, or 256 for N <= 1024); thread t owns rows i = t*EPT .. t*EPT+EPT-1
// (EPT even).  b_{k+1}, b_{k+2} live in registers as (re, im) pairs; v and the step's (2 d, 2 e')
// pairs live in shared memory as float4 holding rows (2p, 2p+1) of thread t at [p][t], so one
// conflict-free 16-byte access serves two rows.  The per-step coefficient and rotation arrays
// are written in global memory in exactly that order ("resident order"), so their loads are
// coalesced.  The one-row halo of b_{k+1} crosses lanes by warp shuffles and warps through a
// small double-buffered shared slot array (one __syncthreads per product).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.h"

namespace {

constexpr int RES_MAXNW = 32;
constexpr int RES_MAXL = 128;
constexpr int GAUGE_NT = 1024;
constexpr int GAUGE_MAXC = 10;  // ld <= 10240

struct ResCoef {
  float cr[RES_MAXL + 1];  // c_k = (-i)^k a_k: real for even k, imaginary for odd k
  float ci[RES_MAXL + 1];
};

struct ResShared {
  float2 slot_first[2][RES_MAXNW];
  float2 slot_last[2][RES_MAXNW];
  float red[RES_MAXNW];
};

// Position of row i in resident order (float2 units) for NT threads of EPT rows each.
__host__ __device__ __forceinline__ size_t res_index(int i, int nt, int ept) {
  const int t = i / ept, q = i - t * ept;
  return ((size_t)(q >> 1) * nt + t) * 2 + (q & 1);
}

// Operator data the gauge kernel reads (device pointers of the plan).
struct GaugeArgs {
  int n, M;
  const double* h0d;
  const double* h0o;
  const double* h1d;
  const double* ko;
  const double* scal;  // sa | sb | sc, M each
  double sbeta;
};

// ---------------------------------------------------------------------------- gauge
// Omega~[k+1][k] = sa_m H0[k+1][k] + i sc_m [H0,H1][k+1][k]  (k < n-1, else 0)
__device__ __forceinline__ void offdiag(const GaugeArgs& p, int m, int k, double& er, double& ei) {
  if (k + 1 < p.n) {
    er = p.scal[m] * p.h0o[k];
    ei = p.scal[2 * p.M + m] * p.ko[k];
  } else {
    er = 0.0;
    ei = 0.0;
  }
}

// phi_k = arg(e_k) reduced to (-pi/2, pi/2], so that e_k e^{-i phi_k} is real (+-|e_k|).
__device__ __forceinline__ double reduced_arg(double er, double ei) {
  if (er == 0.0) return ei == 0.0 ? 0.0 : 0.5 * 3.14159265358979323846;
  return atan(ei / er);
}

// Block-wide exclusive prefix of per-thread chunk sums (GAUGE_NT threads).
__device__ double block_exclusive_scan(double x, double* sw) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    double y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) sw[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    double w = lane < GAUGE_NT / 32 ? sw[lane] : 0.0;
    double wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      double y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    sw[32 + lane] = wi - w;  // exclusive warp offsets
  }
  __syncthreads();
  const double r = sw[32 + warp] + incl - x;
  __syncthreads();
  return r;
}

// theta_k = sum_{j<k} phi_j for k in this thread's chunk [C t, C t + C) of step m (0 if m < 0).
__device__ void phases(const GaugeArgs& p, int m, int ld, int C, double (&th)[GAUGE_MAXC], double* sw) {
  const int k0 = threadIdx.x * C;
  double ph[GAUGE_MAXC];
  double local = 0.0;
#pragma unroll
  for (int q = 0; q < GAUGE_MAXC; ++q) {
    double v = 0.0;
    const int k = k0 + q;
    if (m >= 0 && q < C && k < ld) {
      double er, ei;
      offdiag(p, m, k, er, ei);
      v = reduced_arg(er, ei);
    }
    ph[q] = v;
    local += v;
  }
  double run = block_exclusive_scan(local, sw);
#pragma unroll
  for (int q = 0; q < GAUGE_MAXC; ++q) {
    th[q] = run;
    run += ph[q];
  }
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

template <int NT, int EPT>
struct Resident {
  static constexpr int NW = NT / 32;
  static constexpr int NP = EPT / 2;
  float4* v;   // [NP][NT] state in the step's frame, rows (2p, 2p+1)
  float4* cf;  // [NP][NT] (2 d, 2 e') of rows (2p, 2p+1), e'_i = Omega'[i+1][i]
  ResShared* sh;
  int t, lane, warp;

  // halo of x: left = x[t*EPT - 1], right = x[t*EPT + EPT]
  __device__ __forceinline__ void halo(const float2 (&x)[EPT], int par, float2& left, float2& right) {
    float lr = __shfl_up_sync(0xffffffffu, x[EPT - 1].x, 1);
    float li = __shfl_up_sync(0xffffffffu, x[EPT - 1].y, 1);
    float rr = __shfl_down_sync(0xffffffffu, x[0].x, 1);
    float ri = __shfl_down_sync(0xffffffffu, x[0].y, 1);
    if (lane == 31) sh->slot_last[par][warp] = x[EPT - 1];
    if (lane == 0) sh->slot_first[par][warp] = x[0];
    __syncthreads();
    if (lane == 0) {
      float2 w = warp > 0 ? sh->slot_last[par][warp - 1] : f2(0.f, 0.f);
      lr = w.x;
      li = w.y;
    }
    if (lane == 31) {
      float2 w = warp < NW - 1 ? sh->slot_first[par][warp + 1] : f2(0.f, 0.f);
      rr = w.x;
      ri = w.y;
    }
    left = f2(lr, li);
    right = f2(rr, ri);
  }

  // one row: out = c v + scale (2 Omega' x)_row - out on the (re, im) pair
  __device__ __forceinline__ float2 row(float2 xm, float2 x0, float2 xp, float2 o, float2 vv, float dq, float elo,
                                        float ehi, float cc, bool imag) {
    // c v: a real c scales (re, im); an imaginary c = i cc maps (re, im) to cc (-im, re)
    float2 acc = imag ? f2(-cc * vv.y, cc * vv.x) : f2(cc * vv.x, cc * vv.y);
    acc = __ffma2_rn(f2(-1.f, -1.f), o, acc);
    acc = __ffma2_rn(f2(dq, dq), x0, acc);
    acc = __ffma2_rn(f2(elo, elo), xm, acc);
    acc = __ffma2_rn(f2(ehi, ehi), xp, acc);
    return acc;
  }

  // out = c v + scale (2 Omega') x - out for all rows of the thread.
  // c = (cr, ci) is real (ci = 0) or imaginary (cr = 0).
  __device__ __forceinline__ void apply(const float2 (&x)[EPT], float2 (&out)[EPT], float cr, float ci,
                                        float scale, float el0, int par) {
    float2 left, right;
    halo(x, par, left, right);
    const bool imag = ci != 0.f;
    const float cc = imag ? ci : cr;
    float elo = el0 * scale;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const int s = p * NT + t;
      const float4 c = cf[s];
      const float4 vv = v[s];
      const int q = 2 * p;
      const float d0 = c.x * scale, e0 = c.y * scale, d1 = c.z * scale, e1 = c.w * scale;
      out[q] = row(q == 0 ? left : x[q - 1], x[q], x[q + 1], out[q], lo2(vv), d0, elo, e0, cc, imag);
      out[q + 1] = row(x[q], x[q + 1], q + 1 == EPT - 1 ? right : x[q + 2], out[q + 1], hi2(vv), d1, e0, e1, cc,
                       imag);
      elo = e1;
    }
  }
};

template <int NT, int EPT>
__global__ void __launch_bounds__(NT, 1)
k_tri_resident(const float4* __restrict__ cf_all, const float4* __restrict__ rot_all, int n, int L, int nsteps,
               const double2* __restrict__ x0, double2* __restrict__ xout, int transpose_out, ResCoef coef,
               float ph_re, float ph_im, float clenshaw_bound, unsigned int* status) {
  using Res = Resident<NT, EPT>;
  constexpr int NP = EPT / 2, NW = NT / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Res R;
  float4* base = reinterpret_cast<float4*>(smem_raw);
  R.v = base;
  R.cf = base + NP * NT;
  R.sh = reinterpret_cast<ResShared*>(base + 2 * NP * NT);
  R.t = threadIdx.x;
  R.lane = threadIdx.x & 31;
  R.warp = threadIdx.x >> 5;
  const int t = threadIdx.x;
  const int j = blockIdx.x;  // state index
  const int i0 = t * EPT;
  const size_t stride = (size_t)NP * NT;  // one step of cf / rot, in float4

  // initial state and its squared norm (unitarity bounds every later entry by it)
  float nrm = 0.f;
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    float w[4];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int i = i0 + 2 * p + r;
      float a = 0.f, b = 0.f;
      if (i < n) {
        if (x0) {
          double2 z = x0[(size_t)j * n + i];
          a = (float)z.x;
          b = (float)z.y;
        } else {
          a = i == j ? 1.f : 0.f;
        }
      }
      w[2 * r] = a;
      w[2 * r + 1] = b;
      nrm = fmaf(a, a, fmaf(b, b, nrm));
    }
    R.v[p * NT + t] = make_float4(w[0], w[1], w[2], w[3]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
  if (R.lane == 0) R.sh->red[R.warp] = nrm;
  __syncthreads();
  float tot = 0.f;
#pragma unroll
  for (int w = 0; w < NW; ++w) tot += R.sh->red[w];
  const float bound2 = tot * 1.002f + 1e-30f;
  // |b_k| <= sum_j |c_j| |U_{j-k}(Omega')| |v| <= sum_j (j+1)|a_j| |v| while the spectrum of
  // Omega' lies in [-1, 1] (|U_n| <= n+1 there); outside it U_n grows exponentially.
  const float bcl2 = tot * clenshaw_bound * clenshaw_bound * 1.01f + 1e-30f;
  bool bad = false;

  float2 bA[EPT], bB[EPT];
  for (int m = 0; m < nsteps; ++m) {
    const size_t off = (size_t)m * stride;
    // this step's (2 d, 2 e') and the frame change D_m^+ D_{m-1} of the state (coalesced)
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const int s = p * NT + t;
      const float4 c = cf_all[off + s];
      const float4 r = rot_all[off + s];
      R.cf[s] = c;
      const float4 w = R.v[s];
      R.v[s] = make_float4(r.x * w.x - r.y * w.y, r.x * w.y + r.y * w.x, r.z * w.z - r.w * w.w,
                           r.z * w.w + r.w * w.z);
    }
    // left neighbour's e' (last row of thread t-1)
    const float el0 = t > 0 ? cf_all[off + (size_t)(NP - 1) * NT + t - 1].w : 0.f;
    // b_L = c_L v ; b_{L+1} = 0
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const float4 w = R.v[p * NT + t];
      bA[2 * p] = f2(coef.cr[L] * w.x - coef.ci[L] * w.y, coef.cr[L] * w.y + coef.ci[L] * w.x);
      bA[2 * p + 1] = f2(coef.cr[L] * w.z - coef.ci[L] * w.w, coef.cr[L] * w.w + coef.ci[L] * w.z);
      bB[2 * p] = f2(0.f, 0.f);
      bB[2 * p + 1] = f2(0.f, 0.f);
    }
    int k = L - 1;
    int par = 0;
    // b_k = c_k v + 2 Omega' b_{k+1} - b_{k+2}, two per iteration so the roles stay static
    while (k >= 2) {
      R.apply(bA, bB, coef.cr[k], coef.ci[k], 1.f, el0, par);
      par ^= 1;
      --k;
      R.apply(bB, bA, coef.cr[k], coef.ci[k], 1.f, el0, par);
      par ^= 1;
      --k;
    }
    if (k == 1) {
      R.apply(bA, bB, coef.cr[1], coef.ci[1], 1.f, el0, par);
      par ^= 1;
#pragma unroll
      for (int q = 0; q < EPT; ++q) bad |= !(bB[q].x * bB[q].x + bB[q].y * bB[q].y <= bcl2);
      // b_1 in B, b_2 in A: sum = c_0 v + Omega' b_1 - b_2 (stored operator is 2 Omega')
      R.apply(bB, bA, coef.cr[0], coef.ci[0], 0.5f, el0, par);
#pragma unroll
      for (int q = 0; q < EPT; ++q) bB[q] = bA[q];
    } else {
#pragma unroll
      for (int q = 0; q < EPT; ++q) bad |= !(bA[q].x * bA[q].x + bA[q].y * bA[q].y <= bcl2);
      R.apply(bA, bB, coef.cr[0], coef.ci[0], 0.5f, el0, par);
    }
    // X_m = e^{-i beta h} sum (in B, this step's frame); v <- X_m
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const float2 a = bB[2 * p], b = bB[2 * p + 1];
      const float4 x = make_float4(ph_re * a.x - ph_im * a.y, ph_re * a.y + ph_im * a.x, ph_re * b.x - ph_im * b.y,
                                   ph_re * b.y + ph_im * b.x);
      bad |= !(x.x * x.x + x.y * x.y <= bound2) || !(x.z * x.z + x.w * x.w <= bound2);
      R.v[p * NT + t] = x;
    }
    // the halo slots of the next step's first product use parity 0 again; make sure every
    // warp has consumed this step's last slots before they are overwritten
    __syncthreads();
  }
  // back to the original frame: X = D_last v; unitarity check on the state's norm (a spectral
  // bound that is too tight keeps the entries small but makes the truncated series non-unitary)
  float nrm_end = 0.f;
  const size_t offr = (size_t)nsteps * stride;
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const int s = p * NT + t;
    const float4 r = rot_all[offr + s];
    const float4 w = R.v[s];
    const float4 x = make_float4(r.x * w.x - r.y * w.y, r.x * w.y + r.y * w.x, r.z * w.z - r.w * w.w,
                                 r.z * w.w + r.w * w.z);
    R.v[s] = x;
    nrm_end = fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, fmaf(x.w, x.w, nrm_end))));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nrm_end += __shfl_xor_sync(0xffffffffu, nrm_end, o);
  __syncthreads();
  if (R.lane == 0) R.sh->red[R.warp] = nrm_end;
  __syncthreads();
  float tot_end = 0.f;
#pragma unroll
  for (int w = 0; w < NW; ++w) tot_end += R.sh->red[w];
  bad |= !(fabsf(tot_end - tot) <= 1e-3f * tot + 1e-30f);
  if (bad) atomicOr(status, FQ_BIT_BOUND);
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const float4 w = R.v[p * NT + t];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int i = i0 + 2 * p + r;
      if (i < n) {
        const double2 x = r == 0 ? make_double2((double)w.x, (double)w.y) : make_double2((double)w.z, (double)w.w);
        if (transpose_out) xout[(size_t)i * n + j] = x;
        else xout[(size_t)j * n + i] = x;
      }
    }
  }
}

template <int NT, int EPT>
fq_status launch_cfg(const fq_plan* p, const float4* cf, const float4* rot, const double* x0, double* x,
                     int transpose_out, int nc, int nsteps, const ResCoef& coef, float bcl, cudaStream_t s) {
  const size_t smem = sizeof(float4) * EPT * NT + sizeof(ResShared);
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e =
        cudaFuncSetAttribute(k_tri_resident<NT, EPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return fq_cuda_fail(e, "resident kernel smem attribute");
    attr_done = true;
  }
  k_tri_resident<NT, EPT><<<nc, NT, smem, s>>>(cf, rot, p->n, p->L, nsteps, (const double2*)x0, (double2*)x,
                                                transpose_out, coef, (float)p->phase_re, (float)p->phase_im, bcl,
                                                p->d_status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fq_cuda_fail(e, "resident kernel launch");
  return FQ_OK;
}

// (threads, rows per thread) for dimension n; 0 threads if the resident kernel does not apply.
// 512 x 20 keeps b_{k+1}, b_{k+2} of 20 rows in 124 registers without spills (1024 x 10 would
// have to fit in 64 registers and spills).
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
