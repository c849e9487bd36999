// Second propagation round (§3, last paragraph; §7): period averages of an observable along the
// chain (and, below, the overlap phase error of Eq. 20),  <A>_T = (1/T) int_0^T <psi(t)|A(t)|psi(t)> dt  (Eq. 17),
// for A(t) = a0 H0 + (a1 + s f(t)) H1 (A = H(t) for a0 = 1, a1 = 0, s = 1), evaluated at the
// step boundaries t_m = m h with composite Simpson weights (trapezoid for odd M).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <vector>

#include "internal.h"

namespace {

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;  // valid in thread 0
}

// acc[r] += w <x_r| c0 H0 + c1 H1 |x_r>, tridiagonal H0 (diag, off), diagonal H1; one CTA per row.
__global__ void k_expect_tri(const double2* __restrict__ x, int n, const double* __restrict__ h0d,
                             const double* __restrict__ h0o, const double* __restrict__ h1d, double c0, double c1,
                             double w, double* acc) {
  __shared__ double red[32];
  const double2* row = x + (size_t)blockIdx.x * n;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double2 xi = row[i];
    const double d = c0 * h0d[i] + c1 * h1d[i];
    double yr = d * xi.x, yi = d * xi.y;
    if (i > 0) {
      const double2 xl = row[i - 1];
      yr += c0 * h0o[i - 1] * xl.x;
      yi += c0 * h0o[i - 1] * xl.y;
    }
    if (i + 1 < n) {
      const double2 xr = row[i + 1];
      yr += c0 * h0o[i] * xr.x;
      yi += c0 * h0o[i] * xr.y;
    }
    s += xi.x * yr + xi.y * yi;  // Re(conj(x_i) y_i)
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) acc[blockIdx.x] += w * s;
}

// acc[r] += w <x_r| c0 H0 + c1 H1 |x_r>, dense real-symmetric H0, H1; one CTA per row, the row of
// x staged in shared memory.
__global__ void k_expect_dense(const double2* __restrict__ x, int n, const double* __restrict__ h0,
                               const double* __restrict__ h1, double c0, double c1, double w, double* acc) {
  extern __shared__ double2 xs[];
  __shared__ double red[32];
  const double2* row = x + (size_t)blockIdx.x * n;
  for (int k = threadIdx.x; k < n; k += blockDim.x) xs[k] = row[k];
  __syncthreads();
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double* a = h0 + (size_t)i * n;
    const double* b = h1 + (size_t)i * n;
    double yr = 0.0, yi = 0.0;
    for (int k = 0; k < n; ++k) {
      const double hk = c0 * a[k] + c1 * b[k];
      yr = fma(hk, xs[k].x, yr);
      yi = fma(hk, xs[k].y, yi);
    }
    s += xs[i].x * yr + xs[i].y * yi;
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) acc[blockIdx.x] += w * s;
}

// sigma[r] = |1 - e^{i eps_r T} <phi_r|moved_r>| (Eq. 20, reading R14), one CTA per state row.
__global__ void k_overlap_sigma(const double2* __restrict__ phi, const double2* __restrict__ moved, int n,
                                const double* __restrict__ eps, double period, double* __restrict__ sigma) {
  __shared__ double red[32];
  const double2* a = phi + (size_t)blockIdx.x * n;
  const double2* b = moved + (size_t)blockIdx.x * n;
  double sr = 0.0, si = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const double2 x = a[k], y = b[k];
    sr = fma(x.x, y.x, fma(x.y, y.y, sr));   // Re(conj(x) y)
    si = fma(x.x, y.y, fma(-x.y, y.x, si));  // Im(conj(x) y)
  }
  sr = block_sum(sr, red);
  __syncthreads();
  si = block_sum(si, red);
  if (threadIdx.x == 0) {
    double sn, cs;
    sincos(eps[blockIdx.x] * period, &sn, &cs);
    const double zr = 1.0 - (cs * sr - sn * si), zi = -(cs * si + sn * sr);
    sigma[blockIdx.x] = hypot(zr, zi);
  }
}

__global__ void k_scale_out(const double* acc, int nc, double s, double* out) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nc; q += gridDim.x * blockDim.x) out[q] = s * acc[q];
}

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

extern "C" size_t floquet_observable_workspace_size(const fq_plan* p, int32_t ncols) {
  if (!p || ncols < 1) return 0;
  return up256((size_t)ncols * p->n * 16) + up256((size_t)ncols * 8) + floquet_workspace_size(p, ncols);
}

static fq_status floquet_average_observable_body(fq_plan* p, const void* d_X0, int32_t ncols, double a0, double a1,
                                                 double s_drive, double* d_avg, void* d_ws, size_t ws_bytes,
                                                 void* stream) {
  if (!p || !d_X0 || !d_avg || ncols < 1) {
    fq_set_error("floquet_average_observable: bad arguments");
    return FQ_EINVAL;
  }
  if (p->drive_kind != FQ_DRIVE_COS) {
    fq_set_error("floquet_average_observable: needs a cosine drive plan");
    return FQ_EUNSUPPORTED;
  }
  if (p->format == FQ_DENSE && p->n > 8192) {
    fq_set_error("floquet_average_observable: dense N <= 8192");
    return FQ_EUNSUPPORTED;
  }
  const size_t need = floquet_observable_workspace_size(p, ncols);
  if (!d_ws || ws_bytes < need || ((uintptr_t)d_ws & 255)) {
    fq_set_error("floquet_average_observable: workspace must be >= %zu bytes, 256-byte aligned", need);
    return FQ_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int n = p->n, M = p->steps;
  char* b = (char*)d_ws;
  double* X = (double*)b;
  double* acc = (double*)(b + up256((size_t)ncols * n * 16));
  void* inner = b + up256((size_t)ncols * n * 16) + up256((size_t)ncols * 8);
  const size_t inner_bytes = ws_bytes - up256((size_t)ncols * n * 16) - up256((size_t)ncols * 8);
  cudaError_t e = cudaMemcpyAsync(X, d_X0, (size_t)ncols * n * 16, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, (size_t)ncols * 8, s);
  if (e != cudaSuccess) return fq_cuda_fail(e, "observable setup");
  const double h = p->h;
  std::vector<double> w(M + 1, h);
  if (M % 2 == 0) {
    for (int m = 1; m < M; ++m) w[m] = (m & 1) ? 4.0 * h / 3.0 : 2.0 * h / 3.0;
    w[0] = w[M] = h / 3.0;
  } else {
    w[0] = w[M] = 0.5 * h;
  }
  auto observe = [&](int m) {
    const double t = m * h;
    const double f = fq_drive_f(0, p->f_dc, p->f_ac, p->omega, p->phi0, t);
    const double c0 = a0, c1 = a1 + s_drive * f;
    if (p->format == FQ_TRIDIAG)
      k_expect_tri<<<ncols, 256, 0, s>>>((const double2*)X, n, p->d_h0, p->d_h0o, p->d_h1, c0, c1, w[m], acc);
    else
      k_expect_dense<<<ncols, 256, (size_t)n * sizeof(double2), s>>>((const double2*)X, n, p->d_h0, p->d_h1, c0, c1,
                                                                      w[m], acc);
  };
  if (p->format == FQ_DENSE) {
    e = cudaFuncSetAttribute(k_expect_dense, cudaFuncAttributeMaxDynamicSharedMemorySize, n * (int)sizeof(double2));
    if (e != cudaSuccess) return fq_cuda_fail(e, "observable smem attribute");
  }
  observe(0);
  for (int m = 0; m < M; ++m) {
    fq_status st = floquet_propagate(p, X, X, ncols, m, m + 1, inner, inner_bytes, stream);
    if (st != FQ_OK) return st;
    observe(m + 1);
  }
  k_scale_out<<<(ncols + 255) / 256, 256, 0, s>>>(acc, ncols, 1.0 / p->period, d_avg);
  e = cudaGetLastError();
  return e == cudaSuccess ? FQ_OK : fq_cuda_fail(e, "observable kernels");
}

extern "C" fq_status floquet_average_observable(fq_plan* p, const void* d_X0, int32_t ncols, double a0, double a1,
                                                double s_drive, double* d_avg, void* d_ws, size_t ws_bytes,
                                                void* stream) {
  return fq_guard("floquet_average_observable", [&] {
    return floquet_average_observable_body(p, d_X0, ncols, a0, a1, s_drive, d_avg, d_ws, ws_bytes, stream);
  });
}

extern "C" size_t floquet_overlap_workspace_size(const fq_plan* p, int32_t ncols) {
  if (!p || ncols < 1) return 0;
  return up256((size_t)ncols * p->n * 16) + floquet_workspace_size(p, ncols);
}

static fq_status floquet_overlap_phase_error_body(fq_plan* p, const void* d_states, int32_t ncols,
                                                  const double* d_eps, double* d_sigma, void* d_ws, size_t ws_bytes,
                                                  void* stream) {
  if (!p || !d_states || !d_eps || !d_sigma || ncols < 1) {
    fq_set_error("floquet_overlap_phase_error: bad arguments");
    return FQ_EINVAL;
  }
  const size_t need = floquet_overlap_workspace_size(p, ncols);
  if (!d_ws || ws_bytes < need || ((uintptr_t)d_ws & 255)) {
    fq_set_error("floquet_overlap_phase_error: workspace must be >= %zu bytes, 256-byte aligned", need);
    return FQ_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int n = p->n;
  char* b = (char*)d_ws;
  double* moved = (double*)b;
  const size_t head = up256((size_t)ncols * n * 16);
  // U_T phi~ for every state: the plan's whole chain (step h) on the given rows
  fq_status st = floquet_propagate(p, d_states, moved, ncols, 0, p->steps, b + head, ws_bytes - head, stream);
  if (st != FQ_OK) return st;
  k_overlap_sigma<<<ncols, 256, 0, s>>>((const double2*)d_states, (const double2*)moved, n, d_eps, p->period,
                                        d_sigma);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FQ_OK : fq_cuda_fail(e, "overlap kernel");
}

extern "C" fq_status floquet_overlap_phase_error(fq_plan* p, const void* d_states, int32_t ncols, const double* d_eps,
                                                 double* d_sigma, void* d_ws, size_t ws_bytes, void* stream) {
  return fq_guard("floquet_overlap_phase_error", [&] {
    return floquet_overlap_phase_error_body(p, d_states, ncols, d_eps, d_sigma, d_ws, ws_bytes, stream);
  });
}
