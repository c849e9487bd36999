// Real gauge frame of a Hermitian tridiagonal Omega~ (shared by the resident, tiled and band
// tridiagonal kernels).  Omega~[k+1][k] = e_k is complex; with D = diag(e^{i theta_k}) and
// theta_{k+1} - theta_k = phi_k = arg(e_k) reduced to (-pi/2, pi/2], Omega~ = D Omega' D^+ where
// Omega' is real symmetric with off-diagonal e'_k = e_k e^{-i phi_k} = +-|e_k|.  Phases are
// prefix sums over k, formed in FP64 by one CTA of GAUGE_NT threads.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include "dfl.cuh"

namespace {

constexpr int GAUGE_NT = 1024;
constexpr int GAUGE_MAXC = 10;  // ld <= 10240

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

// ---------------------------------------------------------------------------- per-step tables
template <typename T> struct V2;
template <> struct V2<double> { using t = double2; };
template <> struct V2<float> { using t = float2; };
struct dfl2 {
  dfl x, y;
};
template <> struct V2<dfl> { using t = dfl2; };

// FP64 value into the kernel's coefficient type
template <typename T> __device__ __forceinline__ T coeff_of(double x) { return (T)x; }
template <> __device__ __forceinline__ dfl coeff_of<dfl>(double x) { return dfl_of(x); }

// Block s, step m = m_begin + s: cf[s][k] = (2 d_k, 2 e'_k) and rot[s][k] = (cos, sin) theta_k,
// theta_k = sum_{j<k} phi_j, for k < ld (rows >= n: zero operator).  The prefix sum runs over
// chunks of GAUGE_NT rows with a carried offset, so any ld works.
template <typename T>
__global__ void __launch_bounds__(GAUGE_NT) k_gauge_tile(GaugeArgs p, int ld, int m_begin, typename V2<T>::t* cf,
                                                         typename V2<T>::t* rot) {
  __shared__ double sw[64];
  __shared__ double chunk_total;
  const int s = blockIdx.x, m = m_begin + s;
  typename V2<T>::t* cfs = cf + (size_t)s * ld;
  typename V2<T>::t* rts = rot + (size_t)s * ld;
  double carry = 0.0;
  for (int base = 0; base < ld; base += GAUGE_NT) {
    const int k = base + threadIdx.x;
    double er = 0.0, ei = 0.0, ph = 0.0;
    if (k < ld) {
      offdiag(p, m, k, er, ei);
      ph = reduced_arg(er, ei);
    }
    const double th = carry + block_exclusive_scan(ph, sw);
    if (k < ld) {
      const double d = k < p.n ? p.scal[m] * p.h0d[k] + p.scal[p.M + m] * p.h1d[k] - p.sbeta : 0.0;
      double sp, cp, st, ct;
      sincos(ph, &sp, &cp);
      sincos(th, &st, &ct);
      cfs[k] = {coeff_of<T>(2.0 * d), coeff_of<T>(2.0 * (er * cp + ei * sp))};
      rts[k] = {coeff_of<T>(ct), coeff_of<T>(st)};
    }
    if (threadIdx.x == GAUGE_NT - 1) chunk_total = th - carry + ph;
    __syncthreads();
    carry += chunk_total;
    __syncthreads();
  }
}

}  // namespace
