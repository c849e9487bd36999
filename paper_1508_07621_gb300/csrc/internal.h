// Internal declarations shared by the host planner, the orchestration layer and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>
#include <vector>

#include <atomic>
#include <exception>
#include <functional>
#include <new>

#include "floquet.h"

// Status-word bits raised by device checks.
enum : unsigned int { FQ_BIT_BOUND = 1u, FQ_BIT_TIMEOUT = 2u };

// Which kernel family runs the recurrence for a plan.
enum fq_path : int {
  PATH_DENSE_F64 = 0,     // SIMT FP64 tiled complex GEMM per Chebyshev term
  PATH_DENSE_SPLIT = 1,   // tcgen05 BF16 split GEMM per term
  PATH_TRI_STREAM = 2,    // streaming tridiagonal term kernel (FP32 or FP64)
  PATH_TRI_RESIDENT = 3,  // one CTA per state, whole chain on chip (FP32)
  PATH_TRI_TILE = 5,      // one launch per step, each CTA runs a step's L products on a state segment
  PATH_TRI_BAND = 7,      // FQ_OZAKI tridiagonal: the step's band polynomial on tcgen05 in FP64 emulation
  PATH_DENSE_OZAKI = 6,   // tcgen05 FP64 emulation (fixed-point BF16 slices, exact FP32 sums) per term
  PATH_TRI6 = 8,          // 6th-order tridiagonal: heptadiagonal Omega~ per step, streaming FP64 term kernel
};

// Measurement aid (floquet_kernel_timing): CUDA event pairs recorded on the caller's stream around
// each launch of a path's dominant kernel while enabled; the pool of events is reused.
struct fq_ktimer {
  bool on = false, open = false;  // open: a start event is recorded, its stop not yet
  const char* name = "";
  std::vector<cudaEvent_t> ev;    // (start, stop) pairs
  size_t used = 0;                // events recorded since the last read
  cudaError_t err = cudaSuccess;  // first failure since the last read
};

struct fq_plan {
  // problem
  int n = 0, steps = 0, format = 0, precision = 0, drive_kind = 0, stride = 16, L = 0;
  double period = 0, h = 0, tol = 1e-14;
  int cheb_terms = 0;                   // > 0: fixed L (Table 1's timing runs), else L from tol
  double f_dc = 0, f_ac = 0, omega = 0, phi0 = 0;   // cosine drive (observables)
  // bounds of Omega/h (Eq. 11) and Chebyshev data (Eq. 12)
  double e_min = 0, e_max = 0, beta = 0, delta_e = 0, R = 0;
  std::vector<double> cheb;            // a_0 .. a_L
  double phase_re = 1, phase_im = 0;   // e^{-i beta h}
  // per-step Magnus scalars a_m, b_m, c_m and their Omega~ forms
  std::vector<double> ma, mb, mc;
  std::vector<double> sa, sb, sc;      // Omega~_m = sa H0 + sb H1 + sc i[H0,H1] - sbeta 1
  double sbeta = 0;
  int path = PATH_DENSE_F64;
  bool dense_resident = false;   // PATH_DENSE_F64: small-N resident chain (dense_resident.cu)
  // 6th-order scheme: per step 11 coefficients of Omega_m over {H0, H1, K, K0, K1, K00, K01, K10,
  // K11, KK0, KK1} (K = [H0,H1], K0 = [H0,K], K1 = [H1,K], K00 = [H0,K0], K01 = [H0,K1],
  // K10 = [H1,K0], K11 = [H1,K1], KK0 = [K,K0], KK1 = [K,K1]); real for the symmetric ones,
  // the imaginary factor of the antisymmetric ones
  int order = 4;
  std::vector<double> coef6;   // [M][11]
  // tridiagonal plans of order 6: the 11 basis elements as bands of half-width 3, [11][7][n] with
  // element (i, i + d) at [q][d + 3][i] (zero outside the matrix); on the device in d_cm
  std::vector<double> band6;
  double* d_cm = nullptr;      // K0 .. KK1: 8 matrices n*n after d_k (= K)
  int tile_n = 128;          // split path: output tile width of the tensor-core kernel (autotuned)
  int tile_k = 0;            // split path, 64-wide BF16X3 tiles: K elements a stage (32 or 64; 0 = 64)
  int device = 0;
  // device copies (owned by the plan)
  double* d_h0 = nullptr;    // DENSE: n*n      TRIDIAG: diag n
  double* d_h1 = nullptr;    // DENSE: n*n      TRIDIAG: diag n
  double* d_k = nullptr;     // DENSE: [H0,H1] n*n   TRIDIAG: lower off-diagonal of [H0,H1], n-1
  double* d_h0o = nullptr;   // TRIDIAG: off-diagonal of H0, n-1
  double* d_scal = nullptr;  // 3*M: sa | sb | sc
  // dense bounds left to the caller of fq_host_plan (plan creation runs them on the device):
  // extremes of H0 + g H1 for g in [glo, ghi], widened by kmax ||[H0,H1]||_2
  bool dense_bounds_pending = false;
  double dense_glo = 0, dense_ghi = 0, dense_kmax = 0;
  unsigned int* d_status = nullptr;
  // dense split path: per-plan constants prepared once
  void* split = nullptr;
  fq_ktimer* ktimer = nullptr;  // owned; NULL until floquet_kernel_timing
  int grid_cap = 0;  // > 0: CTAs of a persistent split product (while a batch graph captures the plan)
};

// Brackets one launch of a path's dominant kernel with the plan's timing events (no-ops unless
// floquet_kernel_timing enabled them, and on a stream that is capturing a graph).
void fq_ktimer_start(const fq_plan* p, cudaStream_t s, const char* name);
void fq_ktimer_stop(const fq_plan* p, cudaStream_t s);

// thread-local error message
void fq_set_error(const char* fmt, ...);
fq_status fq_cuda_fail(cudaError_t e, const char* what);

// Runs an entry point's body so that no C++ exception unwinds through the C ABI: a failed host
// allocation becomes FQ_ENOMEM, any other exception FQ_EINVAL, each with a message.
template <class F>
fq_status fq_guard(const char* where, F&& body) noexcept {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    fq_set_error("%s: host allocation failed", where);
    return FQ_ENOMEM;
  } catch (const std::exception& e) {
    fq_set_error("%s: %s", where, e.what());
    return FQ_EINVAL;
  } catch (...) {
    fq_set_error("%s: unexpected host exception", where);
    return FQ_EINVAL;
  }
}

// ---------------------------------------------------------------- host planning (plan.cpp)
double fq_drive_f(int deriv, double f_dc, double f_ac, double omega, double phi0, double t);
void fq_bessel_miller(double R, int L, double* out);    // J_0..J_L
int fq_cheb_order(double R, double tol);  // needs 0 <= R <= FQ_R_MAX
// largest R = h Delta E a plan accepts: about R + 300 Chebyshev products per step; beyond it a
// step is too long for its spectral width and more steps per period are the remedy
constexpr double FQ_R_MAX = 16384.0;
void fq_tridiag_extremes(const double* diag, const double* off, int n, double* lo, double* hi);
// the 6th-order basis of a tridiagonal H0 (diag d0, off-diagonal e0) and diagonal H1 (d1) as bands
void fq_tridiag_band6(const double* d0, const double* e0, const double* d1, int n, std::vector<double>& out);
// y = A x for the operator whose extreme eigenvalues are wanted (host vectors of length n)
using fq_matvec = std::function<void(const double* x, double* y)>;
void fq_lanczos_extremes(const fq_matvec& mv, int n, int ksteps, uint64_t seed, double* lo, double* hi);
// Extremes of H0 + g H1 over g in [glo, ghi], widened by kmax ||[H0,H1]||_2 (dense format):
// apply(which, g, x, y) computes y = (H0 + g H1) x (which 0), H0 x (1) or H1 x (2).
using fq_dense_apply = std::function<void(int which, double g, const double* x, double* y)>;
void fq_dense_bounds(int n, double glo, double ghi, double kmax, const fq_dense_apply& apply, double* emin,
                     double* emax);
// everything but device work; with defer_dense_bounds the dense bounds (and what depends on
// them) are left pending for the caller (see fq_plan::dense_bounds_pending)
fq_status fq_host_plan(const fq_problem* p, fq_plan* plan, bool defer_dense_bounds = false);
// margins of computed bounds, then fq_finish_bounds
fq_status fq_finish_computed_bounds(fq_plan* plan, double emin, double emax);
// y = (H0 + g H1) x (which 0), H0 x (1) or H1 x (2) for dense device H0, H1 (kernels.cu)
void fq_launch_symv2(const double* h0, const double* h1, double g, int which, const double* x, double* y, int n,
                     cudaStream_t s);
// beta, Delta E, R, L, a_l, phase and the Omega~ scalars from bounds [emin, emax] of Omega/h;
// FQ_EINVAL unless emin < emax are finite, FQ_EUNSUPPORTED if R = h Delta E > FQ_R_MAX
fq_status fq_finish_bounds(fq_plan* plan, double emin, double emax);
constexpr int FQ_M6_TERMS = 11;

// ---------------------------------------------------------------- kernels (kernels.cu)
struct fq_term {
  int first, last;         // first term (l = 0) / last term (l = L-1) of a step
  double coef0, coef;      // a_0 (first term) and a_{l+1}
  double ph_re, ph_im;     // e^{-i beta h} (last term)
  double bound2;           // |psi|^2 threshold of the device check (entries of unit-norm states)
  unsigned int* status;
};

// state blocks: planar re/im, ncols rows of length ld (>= n)
template <typename T> struct fq_blk { T* re; T* im; };

void fq_launch_load_states(const double* x_interleaved, fq_blk<double> out, int nc, int n, int ld, cudaStream_t s);
void fq_launch_load_states_f32(const double* x_interleaved, fq_blk<float> out, int nc, int n, int ld, cudaStream_t s);
void fq_launch_identity_f64(fq_blk<double> out, int nc, int n, int ld, cudaStream_t s);
void fq_launch_basis_rows(double* x_interleaved, int nc, int n, int j0, cudaStream_t s);
void fq_launch_identity_f32(fq_blk<float> out, int nc, int n, int ld, cudaStream_t s);
void fq_launch_store_states_f64(fq_blk<double> in, double* x, int nc, int n, int ld, cudaStream_t s);
void fq_launch_store_states_f32(fq_blk<float> in, double* x, int nc, int n, int ld, cudaStream_t s);
void fq_launch_store_transpose_f64(fq_blk<double> in, double* u, int n, int ld, cudaStream_t s);
void fq_launch_store_transpose_f32(fq_blk<float> in, double* u, int n, int ld, cudaStream_t s);

void fq_launch_gemm_f64(const double* a, const double* b, double* c, int n, double alpha, double beta,
                        cudaStream_t s);
void fq_launch_omega_dense_f64(const double* h0, const double* h1, const double* k, int n, double sa,
                               double sb, double sc, double sbeta, double* S, double* A, cudaStream_t s);
// 6th order: S = sum of the symmetric terms - sbeta 1, A = sum of the antisymmetric ones; c[11]
// already divided by h Delta E
void fq_launch_omega6_f64(const fq_plan* p, const double* c, double* S, double* A, cudaStream_t s);
void fq_launch_frobenius(const double* a, size_t count, double* out, cudaStream_t s);
void fq_launch_term_dense_f64(const double* S, const double* A, int n, fq_blk<double> cur, fq_blk<double> prev,
                              fq_blk<double> acc, fq_blk<double> out, int nc, const fq_term& t, cudaStream_t s);

// coefficients of scale * Omega~_m for steps m_begin .. m_begin+nsteps-1, each array [nsteps][ld]
void fq_launch_tri_coeffs_f64(const fq_plan* p, int m_begin, int nsteps, double scale, double* d, double* er,
                              double* ei, cudaStream_t s);
void fq_launch_tri_coeffs_f32(const fq_plan* p, int m_begin, int nsteps, double scale, float* d, float* er,
                              float* ei, cudaStream_t s);
// 6th-order tridiagonal plans: Omega~_m's 7 diagonals (re then im, [7][ld] each, element (i, i + d)
// at [d + 3][i]) from the plan's bands and the step's scaled coefficients c (with -sbeta on the
// diagonal), and one streaming FP64 Chebyshev term with them
void fq_launch_omega_band6(const fq_plan* p, const double* c, double* ore, double* oim, int ld, cudaStream_t s);
void fq_launch_term_band6_f64(const double* ore, const double* oim, int n, fq_blk<double> cur, fq_blk<double> prev,
                              fq_blk<double> acc, fq_blk<double> out, int nc, int ld, const fq_term& t,
                              cudaStream_t s);
void fq_launch_term_tri_f64(const double* d, const double* er, const double* ei, int n, fq_blk<double> cur,
                            fq_blk<double> prev, fq_blk<double> acc, fq_blk<double> out, int nc, int ld,
                            const fq_term& t, cudaStream_t s);
void fq_launch_term_tri_f32(const float* d, const float* er, const float* ei, int n, fq_blk<float> cur,
                            fq_blk<float> prev, fq_blk<float> acc, fq_blk<float> out, int nc, int ld,
                            const fq_term& t, cudaStream_t s);

// resident tridiagonal chain (tri_resident.cu)
int fq_resident_supported(int n, int L);
// Tiled tridiagonal chain (tri_tile.cu): FP64 or FP32, any n, L <= 128.
int fq_tile_supported(int L);
// one bounded wait on an mbarrier nobody arrives on, then FQ_BIT_TIMEOUT (kernels.cu)
void fq_launch_wait_probe(unsigned int* status, long long cycles, cudaStream_t s);
// ---------------------------------------------------------------- dense_resident.cu
bool fq_dense_resident_supported(int n, int L);
// doubles in each of the S and A regions the resident chain needs for nsteps steps
size_t fq_dense_resident_omega_count(int n, int nsteps);
// steps [m_begin, m_end) on planar FP64 states x (nc rows of n), in place
fq_status fq_dense_resident_chain(const fq_plan* p, double* xr, double* xi, int nc, int m_begin, int m_end,
                                  double* S, double* A, cudaStream_t s);
size_t fq_tile_workspace(const fq_plan* p, int nc, int nsteps);
// band.cu: FQ_OZAKI tridiagonal chain (one banded tensor-core product per step)
int fq_band_supported(int L);
size_t fq_band_workspace(const fq_plan* p, int nc, int nsteps);
fq_status fq_band_propagate(fq_plan* p, const double* x0, double* x, int nc, int m_begin, int m_end, int identity,
                            int transpose_out, void* ws, cudaStream_t s);
fq_status fq_tile_propagate(fq_plan* p, const double* x0, double* x, int nc, int m_begin, int m_end, int identity,
                            int transpose_out, void* ws, cudaStream_t s);
size_t fq_resident_coeff_bytes(int n, int steps);
// per-step (2 d, 2 e') of the gauge-real operator and the frame rotations, into `coeff`
void fq_launch_gauge_coeffs(const fq_plan* p, int m_begin, int nsteps, void* coeff, cudaStream_t s);
fq_status fq_launch_resident(const fq_plan* p, const void* coeff, const double* x0, double* x, int transpose_out,
                             int nc, int m_begin, int m_end, cudaStream_t s);

// FP64 emulation on the tensor cores (ozaki.cu, ozaki_grad.cu)
size_t fq_grad_ozaki_workspace(const fq_plan* p);
fq_status fq_grad_ozaki(fq_plan* p, const double* d_f, const void* d_W, double* d_loss, double* d_grad, void* d_ws,
                        cudaStream_t s);
// FP64 loss pieces of adjoint.cu: tau partials over the rows of X_M (FP64 planar, stride n) and
// the seed G_M = -tau W / N^2 as rows
void fq_launch_trace_f64(const double* W, const double* xr, const double* xi, int n, double2* partial,
                         cudaStream_t s);
void fq_launch_seed_f64(const double* W, const double2* tau, int n, double* gr, double* gi, cudaStream_t s);
size_t fq_ozaki_workspace(const fq_plan* p, int nc, void* base, void* out);
fq_status fq_ozaki_propagate(fq_plan* p, const double* x0, double* x, int nc, int m_begin, int m_end, int identity,
                             int transpose_out, void* ws, cudaStream_t s);
// split-precision dense path (dense_split.cu)
size_t fq_split_workspace(const fq_plan* p, int nc, void* base, void* out);
// batched scan as one persistent launch (scan.cu): whether the plans qualify, the bytes it needs
// beyond the plans' own workspaces, and the graph (counter reset + the launch) writing d_U[i];
// plan i's workspace at ws + off[i], the scan's region at ws + extra_off
// FP32 rate probe (kernels.cu): one launch of `blocks` CTAs of 256 threads; returns its flop count
double fq_launch_fp32_probe(int packed, int iters, float* out, int blocks, cudaStream_t s);
int fq_scan_eligible(fq_plan* const* plans, int count);
size_t fq_scan_extra_bytes(fq_plan* const* plans, int count);
fq_status fq_scan_graph(fq_plan* const* plans, int count, void* const* d_U, void* ws, const size_t* off,
                        size_t extra_off, cudaGraph_t* graph);
// True the first time it is called on the current device for this flag word (one bit per
// device, devices 0..31): per-device one-time set-up such as kernel attributes, which the
// runtime keeps per device.
inline bool fq_first_on_device(std::atomic<unsigned>& done) {
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned bit = 1u << (dev & 31);
  return (done.fetch_or(bit) & bit) == 0;
}

// SMs of the current device (queried once per device).
inline int fq_sm_count() {
  static std::atomic<int> cache[32];
  int dev = 0;
  cudaGetDevice(&dev);
  int v = cache[dev & 31].load();
  if (v == 0) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) v = 1;
    cache[dev & 31].store(v);
  }
  return v;
}

// Gradient pieces shared by the FP64 and split adjoints (adjoint.cu): tau = sum of partials and
// loss = 1 - |tau|^2 / N^2; grad_m = 2 Re sum_l w_l D_l from per-CTA partials of D_1..D_L.
void fq_launch_loss(const double2* partial, int count, int n, double* loss, double2* tau, cudaStream_t s);
void fq_launch_grad_reduce(const double2* partial, int ncta, int L, double* grad_m, cudaStream_t s);
// floquet_grad on the tensor cores for BF16X3 / BF16X6 plans (adjoint_split.cu).
size_t fq_grad_split_workspace(const fq_plan* p);
fq_status fq_grad_split(fq_plan* p, const double* d_f, const void* d_W, double* d_loss, double* d_grad, void* d_ws,
                        cudaStream_t s);
fq_status fq_split_propagate(fq_plan* p, const double* x0, double* x, int nc, int m_begin, int m_end, int identity,
                             int transpose_out, void* ws, cudaStream_t s);

void fq_launch_defect(const double* u, int n, const int32_t* cols, int k, double* partial, cudaStream_t s);
