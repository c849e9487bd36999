// Real gauge frame of a Hermitian tridiagonal Omega~ (shared by the resident and tiled tridiagonal
// kernels).  Omega~[k+1][k] = e_k is complex; with D = diag(e^{i theta_k}) and
// theta_{k+1} - theta_k = phi_k = arg(e_k) reduced to (-pi/2, pi/2], Omega~ = D Omega' D^+ where
// Omega' is real symmetric with off-diagonal e'_k = e_k e^{-i phi_k} = +-|e_k|.  Phases are
// prefix sums over k, formed in FP64 by one CTA of GAUGE_NT threads.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

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

}  // namespace
