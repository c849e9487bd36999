// Resident tridiagonal chain (FP32): one CTA carries one state through all steps
// m_begin..m_end-1 without touching HBM in between.
//
// Each step applies sum_{k=0}^{L} c_k T_k(Omega~) v with c_k = (-i)^k a_k (Eqs. 10 and 12:
// psi_k = (-i)^k T_k(Omega~) v) by Clenshaw's backward recurrence
//     b_{L+1} = b_{L+2} = 0,  b_k = c_k v + 2 Omega~ b_{k+1} - b_{k+2}  (k = L..1),
//     sum = c_0 v + Omega~ b_1 - b_2,
// which needs the same L products with Omega~ as the forward recurrence of Eq. 10 but only
// two live vectors besides v.  Then X_m = e^{-i beta h} sum.
//
// Layout: 512 threads; thread t owns rows i = t*EPT .. t*EPT+EPT-1 of the state.  b_{k+1},
// b_{k+2} live in registers; v and the step's 2*Omega~ diagonals live in shared memory at
// [q][t] (element q of thread t), so every shared access is a conflict-free row of 32 words.
// The one-row halo of b_{k+1} crosses lanes by warp shuffles and warps through a small
// double-buffered shared slot array (one __syncthreads per product).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.h"

namespace {

constexpr int RES_NT = 512;
constexpr int RES_NW = RES_NT / 32;
constexpr int RES_MAXL = 128;

struct ResCoef {
  float cr[RES_MAXL + 1];  // c_k = (-i)^k a_k
  float ci[RES_MAXL + 1];
};

struct ResShared {
  float2 slot_first[2][RES_NW];
  float2 slot_last[2][RES_NW];
  float red[RES_NW];
};

template <int EPT>
struct Resident {
  float* vr;  // [EPT][NT]
  float* vi;
  float* d;   // 2 Omega~[i][i]
  float* er;  // 2 Omega~[i+1][i]
  float* ei;
  ResShared* sh;
  int t, lane, warp;

  // halo of x: left = x[t*EPT - 1], right = x[t*EPT + EPT]
  __device__ __forceinline__ void halo(const float (&xr)[EPT], const float (&xi)[EPT], int par, float2& left,
                                       float2& right) {
    float lr = __shfl_up_sync(0xffffffffu, xr[EPT - 1], 1);
    float li = __shfl_up_sync(0xffffffffu, xi[EPT - 1], 1);
    float rr = __shfl_down_sync(0xffffffffu, xr[0], 1);
    float ri = __shfl_down_sync(0xffffffffu, xi[0], 1);
    if (lane == 31) sh->slot_last[par][warp] = make_float2(xr[EPT - 1], xi[EPT - 1]);
    if (lane == 0) sh->slot_first[par][warp] = make_float2(xr[0], xi[0]);
    __syncthreads();
    if (lane == 0) {
      float2 v = warp > 0 ? sh->slot_last[par][warp - 1] : make_float2(0.f, 0.f);
      lr = v.x;
      li = v.y;
    }
    if (lane == 31) {
      float2 v = warp < RES_NW - 1 ? sh->slot_first[par][warp + 1] : make_float2(0.f, 0.f);
      rr = v.x;
      ri = v.y;
    }
    left = make_float2(lr, li);
    right = make_float2(rr, ri);
  }

  // y = (2 Omega~ x) ; out = cmul * v + scale * y - other
  __device__ __forceinline__ void apply(const float (&xr)[EPT], const float (&xi)[EPT], float (&or_)[EPT],
                                        float (&oi)[EPT], float cr, float ci, float scale, float2 el0, int par) {
    float2 left, right;
    halo(xr, xi, par, left, right);
    float elr = el0.x, eli = el0.y;
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const int s = q * RES_NT + t;
      const float dq = d[s], ehr = er[s], ehi = ei[s];
      const float xlr = q == 0 ? left.x : xr[q - 1], xli = q == 0 ? left.y : xi[q - 1];
      const float xrr = q == EPT - 1 ? right.x : xr[q + 1], xri = q == EPT - 1 ? right.y : xi[q + 1];
      float yr = dq * xr[q], yi = dq * xi[q];
      yr = fmaf(elr, xlr, fmaf(-eli, xli, yr));
      yi = fmaf(elr, xli, fmaf(eli, xlr, yi));
      yr = fmaf(ehr, xrr, fmaf(ehi, xri, yr));
      yi = fmaf(ehr, xri, fmaf(-ehi, xrr, yi));
      const float v_r = vr[s], v_i = vi[s];
      float nr = fmaf(scale, yr, -or_[q]);
      float ni = fmaf(scale, yi, -oi[q]);
      nr = fmaf(cr, v_r, fmaf(-ci, v_i, nr));
      ni = fmaf(cr, v_i, fmaf(ci, v_r, ni));
      or_[q] = nr;
      oi[q] = ni;
      elr = ehr;
      eli = ehi;
    }
  }
};

template <int EPT>
__global__ void __launch_bounds__(RES_NT, 1)
k_tri_resident(const float* __restrict__ d2, const float* __restrict__ e2r, const float* __restrict__ e2i, int n,
               int ld, int L, int nsteps, const double2* __restrict__ x0, double2* __restrict__ xout,
               int transpose_out, ResCoef coef, float ph_re, float ph_im, float clenshaw_bound,
               unsigned int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Resident<EPT> R;
  float* base = reinterpret_cast<float*>(smem_raw);
  R.vr = base;
  R.vi = base + EPT * RES_NT;
  R.d = base + 2 * EPT * RES_NT;
  R.er = base + 3 * EPT * RES_NT;
  R.ei = base + 4 * EPT * RES_NT;
  R.sh = reinterpret_cast<ResShared*>(base + 5 * EPT * RES_NT);
  R.t = threadIdx.x;
  R.lane = threadIdx.x & 31;
  R.warp = threadIdx.x >> 5;
  const int t = threadIdx.x;
  const int j = blockIdx.x;  // state index
  const int i0 = t * EPT;

  // initial state and its squared norm (bound of every later entry: unitarity)
  float nrm = 0.f;
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const int i = i0 + q;
    float a = 0.f, b = 0.f;
    if (i < n) {
      if (x0) {
        double2 v = x0[(size_t)j * n + i];
        a = (float)v.x;
        b = (float)v.y;
      } else {
        a = i == j ? 1.f : 0.f;
      }
    }
    R.vr[q * RES_NT + t] = a;
    R.vi[q * RES_NT + t] = b;
    nrm = fmaf(a, a, fmaf(b, b, nrm));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
  if (R.lane == 0) R.sh->red[R.warp] = nrm;
  __syncthreads();
  float tot = 0.f;
#pragma unroll
  for (int w = 0; w < RES_NW; ++w) tot += R.sh->red[w];
  const float bound2 = tot * 1.002f + 1e-30f;
  // |b_k| <= sum_j |c_j| |U_{j-k}(Omega~)| |v| <= sum_j (j+1)|a_j| |v| while the spectrum of
  // Omega~ lies in [-1, 1] (|U_n| <= n+1 there); outside it U_n grows exponentially.
  const float bcl2 = tot * clenshaw_bound * clenshaw_bound * 1.01f + 1e-30f;
  bool bad = false;

  float bAr[EPT], bAi[EPT], bBr[EPT], bBi[EPT];
  for (int m = 0; m < nsteps; ++m) {
    // this thread's rows of 2 Omega~_m, plus the left neighbour's off-diagonal
    const size_t off = (size_t)m * ld;
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const int i = i0 + q;
      const bool in = i < ld;
      R.d[q * RES_NT + t] = in ? __ldg(d2 + off + i) : 0.f;
      R.er[q * RES_NT + t] = in ? __ldg(e2r + off + i) : 0.f;
      R.ei[q * RES_NT + t] = in ? __ldg(e2i + off + i) : 0.f;
    }
    const float2 el0 = i0 > 0 && i0 - 1 < ld ? make_float2(__ldg(e2r + off + i0 - 1), __ldg(e2i + off + i0 - 1))
                                             : make_float2(0.f, 0.f);
    // b_L = c_L v ; b_{L+1} = 0
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const int s = q * RES_NT + t;
      const float v_r = R.vr[s], v_i = R.vi[s];
      bAr[q] = coef.cr[L] * v_r - coef.ci[L] * v_i;
      bAi[q] = coef.cr[L] * v_i + coef.ci[L] * v_r;
      bBr[q] = 0.f;
      bBi[q] = 0.f;
    }
    int k = L - 1;
    int par = 0;
    // b_k = c_k v + 2 Omega~ b_{k+1} - b_{k+2}, two per iteration so the roles stay static
    while (k >= 2) {
      R.apply(bAr, bAi, bBr, bBi, coef.cr[k], coef.ci[k], 1.f, el0, par);
      par ^= 1;
      --k;
      R.apply(bBr, bBi, bAr, bAi, coef.cr[k], coef.ci[k], 1.f, el0, par);
      par ^= 1;
      --k;
    }
    if (k == 1) {
      R.apply(bAr, bAi, bBr, bBi, coef.cr[1], coef.ci[1], 1.f, el0, par);
      par ^= 1;
#pragma unroll
      for (int q = 0; q < EPT; ++q) bad |= !(bBr[q] * bBr[q] + bBi[q] * bBi[q] <= bcl2);
      // b_1 in B, b_2 in A: sum = c_0 v + Omega~ b_1 - b_2  (stored operator is 2 Omega~)
      R.apply(bBr, bBi, bAr, bAi, coef.cr[0], coef.ci[0], 0.5f, el0, par);
#pragma unroll
      for (int q = 0; q < EPT; ++q) { bBr[q] = bAr[q]; bBi[q] = bAi[q]; }
    } else {
      // k == 0: b_1 in A, b_2 in B
#pragma unroll
      for (int q = 0; q < EPT; ++q) bad |= !(bAr[q] * bAr[q] + bAi[q] * bAi[q] <= bcl2);
      R.apply(bAr, bAi, bBr, bBi, coef.cr[0], coef.ci[0], 0.5f, el0, par);
    }
    // X_m = e^{-i beta h} sum (now in B); v <- X_m
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const int s = q * RES_NT + t;
      const float xr = ph_re * bBr[q] - ph_im * bBi[q];
      const float xi = ph_re * bBi[q] + ph_im * bBr[q];
      bad |= !(xr * xr + xi * xi <= bound2);
      R.vr[s] = xr;
      R.vi[s] = xi;
    }
    // the halo slots of the next step's first product use parity 0 again; make sure every
    // warp has consumed this step's last slots before they are overwritten
    __syncthreads();
  }
  // unitarity of the chain: the state's norm must be preserved (a spectral bound that is too
  // tight keeps the entries small but makes the truncated series non-unitary)
  float nrm_end = 0.f;
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const int s = q * RES_NT + t;
    nrm_end = fmaf(R.vr[s], R.vr[s], fmaf(R.vi[s], R.vi[s], nrm_end));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nrm_end += __shfl_xor_sync(0xffffffffu, nrm_end, o);
  __syncthreads();
  if (R.lane == 0) R.sh->red[R.warp] = nrm_end;
  __syncthreads();
  float tot_end = 0.f;
#pragma unroll
  for (int w = 0; w < RES_NW; ++w) tot_end += R.sh->red[w];
  bad |= !(fabsf(tot_end - tot) <= 1e-3f * tot + 1e-30f);
  if (bad) atomicOr(status, FQ_BIT_BOUND);
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const int i = i0 + q;
    if (i < n) {
      const int s = q * RES_NT + t;
      const double2 v = make_double2((double)R.vr[s], (double)R.vi[s]);
      if (transpose_out) xout[(size_t)i * n + j] = v;
      else xout[(size_t)j * n + i] = v;
    }
  }
}

template <int EPT>
fq_status launch_ept(const fq_plan* p, const float* d2, const float* e2r, const float* e2i, const double* x0,
                     double* x, int transpose_out, int nc, int nsteps, const ResCoef& coef, float bcl,
                     cudaStream_t s) {
  const int ld = (p->n + 3) & ~3;
  const size_t smem = sizeof(float) * 5 * EPT * RES_NT + sizeof(ResShared);
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(k_tri_resident<EPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return fq_cuda_fail(e, "resident kernel smem attribute");
    attr_done = true;
  }
  k_tri_resident<EPT><<<nc, RES_NT, smem, s>>>(d2, e2r, e2i, p->n, ld, p->L, nsteps, (const double2*)x0,
                                                (double2*)x, transpose_out, coef, (float)p->phase_re,
                                                (float)p->phase_im, bcl, p->d_status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fq_cuda_fail(e, "resident kernel launch");
  return FQ_OK;
}

}  // namespace

static int ept_for(int n) {
  const int need = (n + RES_NT - 1) / RES_NT;
  if (need <= 4) return 4;
  if (need <= 8) return 8;
  if (need <= 12) return 12;
  if (need <= 16) return 16;
  if (need <= 20) return 20;
  return 0;  // 5 * 24 * 512 floats would exceed the 227 KB shared-memory limit

}

int fq_resident_supported(int n, int L) { return ept_for(n) > 0 && L <= RES_MAXL && L >= 1; }

size_t fq_resident_coeff_bytes(int n, int steps) {
  const size_t ld = (size_t)((n + 3) & ~3);
  return 3 * ld * (size_t)steps * sizeof(float);
}

// d2, e2r, e2i: [nsteps][ld] coefficients of 2 Omega~ for the steps to run, in order.
fq_status fq_launch_resident(const fq_plan* p, const float* d2, const float* e2, const double* x0, double* x,
                             int transpose_out, int nc, int m_begin, int m_end, cudaStream_t s) {
  const int ld = (p->n + 3) & ~3;
  const int nsteps = m_end - m_begin;
  const float* e2r = e2;
  const float* e2i = e2 + (size_t)nsteps * ld;
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
  switch (ept_for(p->n)) {
    case 4: return launch_ept<4>(p, d2, e2r, e2i, x0, x, transpose_out, nc, nsteps, coef, (float)bcl, s);
    case 8: return launch_ept<8>(p, d2, e2r, e2i, x0, x, transpose_out, nc, nsteps, coef, (float)bcl, s);
    case 12: return launch_ept<12>(p, d2, e2r, e2i, x0, x, transpose_out, nc, nsteps, coef, (float)bcl, s);
    case 16: return launch_ept<16>(p, d2, e2r, e2i, x0, x, transpose_out, nc, nsteps, coef, (float)bcl, s);
    case 20: return launch_ept<20>(p, d2, e2r, e2i, x0, x, transpose_out, nc, nsteps, coef, (float)bcl, s);
    default: fq_set_error("resident kernel: n = %d too large", p->n); return FQ_EUNSUPPORTED;
  }
}
