// floquet_build_UT_static: U_T through the resident FP32 tridiagonal kernel without any device
// allocation.  For callers that cannot call cudaMalloc - code that runs where another runtime
// owns all device memory, or that must not grow its footprint after start-up.  All scratch
// (operators, per-step scalars, the per-step operator coefficients and frame rotations, and the
// status word) lives in
// one file-scope __device__ array of FLOQUET_STATIC_SCRATCH_BYTES; the caller passes the problem
// (host arrays) and the output.  The kernels are the library's existing ones.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "internal.h"

// 16 MiB on every GPU where the library's device code is loaded, held until the process exits.
// With CUDA's lazy module loading (the default) that happens at the first call on a device, not
// when the library is opened.
static __device__ __align__(256) unsigned char g_fq_static_scratch[FLOQUET_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device address of the scratch array for the current device.  Host code only sees a host-side
// stand-in under the array's name, so the address is looked up once per device, with that
// device current, and cached.
fq_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fq_cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) {
    fq_set_error("floquet_build_UT_static: device %d out of range", dev);
    return FQ_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_fq_static_scratch);
    if (e != cudaSuccess) return fq_cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return FQ_OK;
}

}  // namespace

static fq_status build_static(const fq_problem* prob, void* d_U, void* stream) {
  if (!prob || !d_U) {
    fq_set_error("floquet_build_UT_static: NULL problem or output");
    return FQ_EINVAL;
  }
  if (prob->format != FQ_TRIDIAG || prob->precision != FQ_FP32) {
    fq_set_error("floquet_build_UT_static: only FQ_TRIDIAG with FQ_FP32 (resident kernel)");
    return FQ_EUNSUPPORTED;
  }
  if (prob->kernel != FQ_KERNEL_AUTO && prob->kernel != FQ_KERNEL_RESIDENT) {
    fq_set_error("floquet_build_UT_static: runs the resident kernel only (kernel = %d requested)", (int)prob->kernel);
    return FQ_EUNSUPPORTED;
  }
  fq_plan p;
  fq_status st = fq_host_plan(prob, &p);
  if (st != FQ_OK) return st;
  const int n = p.n, M = p.steps;
  if (!fq_resident_supported(n, p.L)) {
    fq_set_error("floquet_build_UT_static: resident kernel needs N <= 10240 and L <= 128 (N = %d, L = %d)", n, p.L);
    return FQ_EUNSUPPORTED;
  }
  const size_t nm1 = (size_t)(n > 1 ? n - 1 : 1);
  const size_t off_status = 0;
  const size_t off_scal = off_status + 256;
  const size_t off_h0 = off_scal + up256(3 * (size_t)M * sizeof(double));
  const size_t off_h1 = off_h0 + up256((size_t)n * sizeof(double));
  const size_t off_h0o = off_h1 + up256((size_t)n * sizeof(double));
  const size_t off_k = off_h0o + up256(nm1 * sizeof(double));
  const size_t off_coef = off_k + up256(nm1 * sizeof(double));
  const size_t need = off_coef + up256(fq_resident_coeff_bytes(n, M));
  if (need > (size_t)FLOQUET_STATIC_SCRATCH_BYTES) {
    fq_set_error("floquet_build_UT_static: needs %zu bytes of scratch ((2M+1) * %zu padded rows * 8 B + small), "
                 "limit %zu; use floquet_build_UT with a caller workspace",
                 need, fq_resident_coeff_bytes(n, 0) / sizeof(float2), (size_t)FLOQUET_STATIC_SCRATCH_BYTES);
    return FQ_EINVAL;
  }
  void* base = nullptr;
  st = scratch_address(&base);
  if (st != FQ_OK) return st;
  char* b = (char*)base;
  cudaStream_t s = (cudaStream_t)stream;
  p.d_status = (unsigned int*)(b + off_status);
  p.d_scal = (double*)(b + off_scal);
  p.d_h0 = (double*)(b + off_h0);
  p.d_h1 = (double*)(b + off_h1);
  p.d_h0o = (double*)(b + off_h0o);
  p.d_k = (double*)(b + off_k);
  void* coef = b + off_coef;

  // host-side operands for the upload: per-step Omega~ scalars and the commutator diagonal
  std::vector<double> scal(3 * (size_t)M);
  for (int m = 0; m < M; ++m) {
    scal[m] = p.sa[m];
    scal[M + m] = p.sb[m];
    scal[2 * M + m] = p.sc[m];
  }
  std::vector<double> kl(nm1, 0.0);
  for (int i = 0; i + 1 < n; ++i) kl[i] = prob->h0_off[i] * (prob->h1[i] - prob->h1[i + 1]);

  cudaError_t e = cudaMemsetAsync(p.d_status, 0, sizeof(unsigned int), s);  // last call's bits
  if (e == cudaSuccess) e = cudaMemcpyAsync(p.d_scal, scal.data(), scal.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p.d_h0, prob->h0, n * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p.d_h1, prob->h1, n * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && n > 1)
    e = cudaMemcpyAsync(p.d_h0o, prob->h0_off, (n - 1) * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && n > 1) e = cudaMemcpyAsync(p.d_k, kl.data(), (n - 1) * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fq_cuda_fail(e, "floquet_build_UT_static upload");

  fq_launch_gauge_coeffs(&p, 0, M, coef, s);
  st = fq_launch_resident(&p, coef, nullptr, (double*)d_U, 1, n, 0, M, s);
  if (st != FQ_OK) return st;
  // the host vectors above are staged by the copies; wait for the chain and read the check
  unsigned int bits = 0;
  e = cudaMemcpyAsync(&bits, p.d_status, sizeof(bits), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fq_cuda_fail(e, "floquet_build_UT_static");
  if (bits) {
    fq_set_error("device check: an entry exceeded the unitarity bound or was NaN (spectral bounds too tight?)");
    return FQ_EBOUND;
  }
  return FQ_OK;
}

extern "C" fq_status floquet_build_UT_static(const fq_problem* prob, void* d_U, void* stream) {
  return fq_guard("floquet_build_UT_static", [&] { return build_static(prob, d_U, stream); });
}
