// Baseline kernels: layout conversion, Omega~ builds (stage a2), the plain FP64 dense
// Chebyshev-term GEMM (a3), the streaming tridiagonal term (a4) with the Bessel
// accumulation and step close fused into the epilogue (a5, a6), and the unitarity defect (a7).
//
// States are stored planar (re, im planes), one state per row of length ld (>= n), so the
// Chebyshev term Y = Omega~ Psi becomes Y^T = Psi^T Omega~^T: every state row is a
// contiguous vector (the row layout of §5).
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "dense_core.cuh"

namespace {

template <typename T> struct vec2;
template <> struct vec2<double> { using t = double2; };
template <> struct vec2<float> { using t = float2; };

__device__ __forceinline__ void check_bound(double re, double im, const fq_term& t) {
  if (!(re * re + im * im <= t.bound2)) atomicOr(t.status, FQ_BIT_BOUND);
}

// Epilogue shared by every term kernel, for one element with Y = (Omega~ psi_l)[element]:
//  first (l = 0):  psi_1 = -i Y,            acc = a_0 psi_0 + a_1 psi_1
//  middle:         psi_{l+1} = -2i Y + psi_{l-1},  acc += a_{l+1} psi_{l+1}
//  last:           X = e^{-i beta h} (acc + a_L psi_L)   (Eq. 12)
// `cur0` is psi_0 (only read on the first term), `prev` psi_{l-1}.
template <typename T>
__device__ __forceinline__ void term_epilogue(T yr, T yi, T cur_r, T cur_i, const T* prev_re, const T* prev_im,
                                              T* acc_re, T* acc_im, T* out_re, T* out_im, size_t idx,
                                              const fq_term& t) {
  T pr, pi;
  if (t.first) {
    pr = yi;
    pi = -yr;
  } else {
    pr = (T)2 * yi + prev_re[idx];
    pi = (T)-2 * yr + prev_im[idx];
  }
  check_bound((double)pr, (double)pi, t);
  T ar, ai;
  if (t.first) {
    ar = (T)t.coef0 * cur_r + (T)t.coef * pr;
    ai = (T)t.coef0 * cur_i + (T)t.coef * pi;
  } else {
    ar = acc_re[idx] + (T)t.coef * pr;
    ai = acc_im[idx] + (T)t.coef * pi;
  }
  if (t.last) {
    out_re[idx] = (T)t.ph_re * ar - (T)t.ph_im * ai;
    out_im[idx] = (T)t.ph_re * ai + (T)t.ph_im * ar;
  } else {
    out_re[idx] = pr;
    out_im[idx] = pi;
    acc_re[idx] = ar;
    acc_im[idx] = ai;
  }
}

// ------------------------------------------------------------------ layout conversion
template <typename T>
__global__ void k_load_states(const double2* __restrict__ x, T* re, T* im, int nc, int n, int ld) {
  size_t total = (size_t)nc * ld;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    int r = (int)(q / ld), i = (int)(q % ld);
    double2 v = i < n ? x[(size_t)r * n + i] : make_double2(0.0, 0.0);
    re[q] = (T)v.x;
    im[q] = (T)v.y;
  }
}

template <typename T>
__global__ void k_identity(T* re, T* im, int nc, int n, int ld) {
  size_t total = (size_t)nc * ld;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    int r = (int)(q / ld), i = (int)(q % ld);
    re[q] = (T)(i == r ? 1 : 0);
    im[q] = (T)0;
  }
}

// Rows r = 0 .. nc-1 of an interleaved complex128 block are the basis states e_{j0 + r} (the
// columns j0 .. j0+nc-1 of the identity that one rank propagates, §5).
__global__ void k_basis_rows(double2* x, int nc, int n, int j0) {
  const size_t total = (size_t)nc * n;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(q / n), i = (int)(q % n);
    x[q] = make_double2(i == j0 + r ? 1.0 : 0.0, 0.0);
  }
}

template <typename T>
__global__ void k_store_states(const T* __restrict__ re, const T* __restrict__ im, double2* x, int nc, int n, int ld) {
  size_t total = (size_t)nc * n;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    int r = (int)(q / n), i = (int)(q % n);
    x[q] = make_double2((double)re[(size_t)r * ld + i], (double)im[(size_t)r * ld + i]);
  }
}

// U[i][j] = X_j[i]: 32x32 tiles through shared memory so both sides are coalesced.
template <typename T>
__global__ void k_store_transpose(const T* __restrict__ re, const T* __restrict__ im, double2* u, int n, int ld) {
  __shared__ double2 tile[32][33];
  int j0 = blockIdx.y * 32, i0 = blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int j = j0 + r, i = i0 + threadIdx.x;
    if (j < n && i < n) tile[r][threadIdx.x] = make_double2((double)re[(size_t)j * ld + i], (double)im[(size_t)j * ld + i]);
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int i = i0 + r, j = j0 + threadIdx.x;
    if (j < n && i < n) u[(size_t)i * n + j] = tile[threadIdx.x][r];
  }
}

// ------------------------------------------------------------------ dense FP64
// C = alpha * A B + beta * C for row-major n x n (used once per plan for [H0, H1]).
__global__ void k_gemm_f64(const double* __restrict__ a, const double* __restrict__ b, double* c, int n,
                           double alpha, double beta) {
  __shared__ double sa[16][17], sb[16][17];
  int row = blockIdx.y * 16 + threadIdx.y, col = blockIdx.x * 16 + threadIdx.x;
  double s = 0.0;
  for (int k0 = 0; k0 < n; k0 += 16) {
    sa[threadIdx.y][threadIdx.x] = (row < n && k0 + threadIdx.x < n) ? a[(size_t)row * n + k0 + threadIdx.x] : 0.0;
    sb[threadIdx.y][threadIdx.x] = (k0 + threadIdx.y < n && col < n) ? b[(size_t)(k0 + threadIdx.y) * n + col] : 0.0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) s += sa[threadIdx.y][k] * sb[k][threadIdx.x];
    __syncthreads();
  }
  if (row < n && col < n) c[(size_t)row * n + col] = alpha * s + beta * c[(size_t)row * n + col];
}

// Omega~_m = S + i A with S = sa H0 + sb H1 - sbeta 1 (real symmetric) and A = sc [H0,H1]
// (real antisymmetric): Eq. 11 applied to Omega_m/h (stage a2), FP64.
__global__ void k_omega_dense_f64(const double* __restrict__ h0, const double* __restrict__ h1,
                                  const double* __restrict__ k, int n, double sa, double sb, double sc,
                                  double sbeta, double* S, double* A) {
  size_t total = (size_t)n * n;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(q / n), j = (int)(q % n);
    S[q] = sa * h0[q] + sb * h1[q] - (i == j ? sbeta : 0.0);
    A[q] = sc * k[q];
  }
}

// 6th order: Omega~_m = sum_q c_q M_q with M_q over {H0, H1, K, K0, K1, K00, K01, K10, K11, KK0,
// KK1}; the symmetric terms form S (minus sbeta 1), the antisymmetric ones A (Omega~ = S + i A).
struct Omega6Args {
  const double* m[FQ_M6_TERMS];
  double c[FQ_M6_TERMS];
  double sbeta;
  int n;
};

__global__ void k_omega6_f64(Omega6Args a, double* S, double* A) {
  const size_t total = (size_t)a.n * a.n;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(q / a.n), j = (int)(q % a.n);
    double s = (i == j) ? -a.sbeta : 0.0;
    s = fma(a.c[0], a.m[0][q], s);
    s = fma(a.c[1], a.m[1][q], s);
    s = fma(a.c[3], a.m[3][q], s);
    s = fma(a.c[4], a.m[4][q], s);
    s = fma(a.c[9], a.m[9][q], s);
    s = fma(a.c[10], a.m[10][q], s);
    double t = a.c[2] * a.m[2][q];
    t = fma(a.c[5], a.m[5][q], t);
    t = fma(a.c[6], a.m[6][q], t);
    t = fma(a.c[7], a.m[7][q], t);
    t = fma(a.c[8], a.m[8][q], t);
    S[q] = s;
    A[q] = t;
  }
}

__global__ void k_frobenius(const double* __restrict__ a, size_t count, double* out) {
  __shared__ double red[256];
  double s = 0.0;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < count; q += (size_t)gridDim.x * blockDim.x)
    s = fma(a[q], a[q], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, red[0]);
}

// One Chebyshev term, dense FP64: Y^T[j][i] = sum_k Psi[j][k] (S[i][k] + i A[i][k]) (tile loop in
// dense_core.cuh) followed by the fused recurrence / Bessel accumulation / step-close epilogue.
// A == nullptr selects the real-operator variant (piecewise drives: c_m = 0).
template <int BJ, int BI, int BK, int TJ, int TI, bool HAS_A>
__global__ void __launch_bounds__((BJ / TJ) * (BI / TI))
k_term_dense_f64(const double* __restrict__ S, const double* __restrict__ A, int n,
                 const double* __restrict__ cur_re, const double* __restrict__ cur_im,
                 const double* prev_re, const double* prev_im, double* acc_re, double* acc_im,
                 double* out_re, double* out_im, int nc, fq_term t) {
  constexpr int NTX = BI / TI;
  const int tx = threadIdx.x % NTX, ty = threadIdx.x / NTX;
  const int j0 = blockIdx.y * BJ, i0 = blockIdx.x * BI;
  double yr[TJ][TI], yi[TJ][TI];
  dense_tile_f64<BJ, BI, BK, TJ, TI, HAS_A>(S, A, n, cur_re, cur_im, nc, j0, i0, yr, yi);
#pragma unroll
  for (int u = 0; u < TJ; ++u)
#pragma unroll
    for (int v = 0; v < TI; ++v) {
      int j = j0 + ty * TJ + u, i = i0 + tx * TI + v;
      if (j < nc && i < n) {
        size_t idx = (size_t)j * n + i;
        double c0r = t.first ? cur_re[idx] : 0.0, c0i = t.first ? cur_im[idx] : 0.0;
        term_epilogue<double>(yr[u][v], yi[u][v], c0r, c0i, prev_re, prev_im, acc_re, acc_im, out_re, out_im,
                              idx, t);
      }
    }
}

// ------------------------------------------------------------------ tridiagonal
// Per-step coefficients of scale * Omega~_m for every step, stage a2 in FP64 arithmetic:
//  d[m][i]  = scale (sa_m H0[i][i] + sb_m H1[i][i] - sbeta)
//  e[m][i]  = scale (sa_m H0[i+1][i] + i sc_m [H0,H1][i+1][i])     (Omega~[i+1][i]; Omega~[i][i+1] = conj)
// Entries i >= n (d) and i >= n-1 (e) are zero so padded rows stay zero.
template <typename T>
__global__ void k_tri_coeffs(const double* __restrict__ h0d, const double* __restrict__ h0o,
                             const double* __restrict__ h1d, const double* __restrict__ ko,
                             const double* __restrict__ scal, int n, int ld, int M, int m_begin, int nsteps,
                             double sbeta, double scale, T* d, T* er, T* ei) {
  size_t total = (size_t)nsteps * ld;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    int m = m_begin + (int)(q / ld), i = (int)(q % ld);
    double sa = scal[m], sb = scal[M + m], sc = scal[2 * M + m];
    d[q] = (T)(i < n ? scale * (sa * h0d[i] + sb * h1d[i] - sbeta) : 0.0);
    er[q] = (T)(i + 1 < n ? scale * sa * h0o[i] : 0.0);
    ei[q] = (T)(i + 1 < n ? scale * sc * ko[i] : 0.0);
  }
}

// Streaming tridiagonal term: every element reads psi_l with its two neighbours, psi_{l-1} and
// acc, and writes psi_{l+1} (in place of psi_{l-1}) and acc.  4 consecutive elements per
// thread; rows are padded to ld (multiple of 4) with zeros.  All loads of a thread are issued
// before any arithmetic (16-byte vector loads), so each thread pays one memory round trip.
template <typename T> struct Quad;
template <> struct Quad<float> {
  static __device__ __forceinline__ void load(const float* p, float (&v)[4]) {
    float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  }
  static __device__ __forceinline__ void store(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <> struct Quad<double> {
  static __device__ __forceinline__ void load(const double* p, double (&v)[4]) {
    double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
  static __device__ __forceinline__ void store(double* p, const double (&v)[4]) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
};

template <typename T>
__global__ void __launch_bounds__(256)
k_term_tri(const T* __restrict__ d, const T* __restrict__ er, const T* __restrict__ ei, int ld,
           const T* __restrict__ cur_re, const T* __restrict__ cur_im, const T* prev_re, const T* prev_im,
           T* acc_re, T* acc_im, T* out_re, T* out_im, fq_term t) {
  const int j = blockIdx.y;
  const int i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (i0 >= ld) return;
  const size_t row = (size_t)j * ld;
  T cr[4], ci[4], dd[4], lr[4], li[4], pr[4], pi[4], ar[4], ai[4];
  Quad<T>::load(cur_re + row + i0, cr);
  Quad<T>::load(cur_im + row + i0, ci);
  Quad<T>::load(d + i0, dd);
  Quad<T>::load(er + i0, lr);
  Quad<T>::load(ei + i0, li);
  const T cl_r = i0 > 0 ? cur_re[row + i0 - 1] : (T)0, cl_i = i0 > 0 ? cur_im[row + i0 - 1] : (T)0;
  const T cx_r = i0 + 4 < ld ? cur_re[row + i0 + 4] : (T)0, cx_i = i0 + 4 < ld ? cur_im[row + i0 + 4] : (T)0;
  const T el_r = i0 > 0 ? er[i0 - 1] : (T)0, el_i = i0 > 0 ? ei[i0 - 1] : (T)0;
  if (!t.first) {
    Quad<T>::load(prev_re + row + i0, pr);
    Quad<T>::load(prev_im + row + i0, pi);
    Quad<T>::load(acc_re + row + i0, ar);
    Quad<T>::load(acc_im + row + i0, ai);
  }
  T o_r[4], o_i[4], a_r[4], a_i[4];
  bool bad = false;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const T xlr = q == 0 ? cl_r : cr[q - 1], xli = q == 0 ? cl_i : ci[q - 1];
    const T xrr = q == 3 ? cx_r : cr[q + 1], xri = q == 3 ? cx_i : ci[q + 1];
    const T elr = q == 0 ? el_r : lr[q - 1], eli = q == 0 ? el_i : li[q - 1];
    // y = d_i x_i + e_{i-1} x_{i-1} + conj(e_i) x_{i+1}
    T yr = dd[q] * cr[q], yi = dd[q] * ci[q];
    yr = fma(elr, xlr, fma(-eli, xli, yr));
    yi = fma(elr, xli, fma(eli, xlr, yi));
    yr = fma(lr[q], xrr, fma(li[q], xri, yr));
    yi = fma(lr[q], xri, fma(-li[q], xrr, yi));
    T nr, ni, sr, si;
    if (t.first) {
      nr = yi;
      ni = -yr;
      sr = (T)t.coef0 * cr[q] + (T)t.coef * nr;
      si = (T)t.coef0 * ci[q] + (T)t.coef * ni;
    } else {
      nr = (T)2 * yi + pr[q];
      ni = (T)-2 * yr + pi[q];
      sr = ar[q] + (T)t.coef * nr;
      si = ai[q] + (T)t.coef * ni;
    }
    bad |= !(nr * nr + ni * ni <= (T)t.bound2);  // in T: FP64 arithmetic runs far below the FP32 rate on sm_103
    if (t.last) {
      o_r[q] = (T)t.ph_re * sr - (T)t.ph_im * si;
      o_i[q] = (T)t.ph_re * si + (T)t.ph_im * sr;
    } else {
      o_r[q] = nr;
      o_i[q] = ni;
      a_r[q] = sr;
      a_i[q] = si;
    }
  }
  if (bad) atomicOr(t.status, FQ_BIT_BOUND);
  Quad<T>::store(out_re + row + i0, o_r);
  Quad<T>::store(out_im + row + i0, o_i);
  if (!t.last) {
    Quad<T>::store(acc_re + row + i0, a_r);
    Quad<T>::store(acc_im + row + i0, a_i);
  }
}

// ------------------------------------------------------------------ 6th-order tridiagonal plans
// Omega~_m = sum_q c_q B_q - sbeta 1 over the 11 basis bands (Eq. 14 in full, reading R12): the
// symmetric elements give the real part S, the antisymmetric ones (whose coefficient is the
// imaginary factor) the imaginary part A, so Omega~ = S + i A is Hermitian.  Diagonal d + 3 of
// the output holds (i, i + d); rows i >= n are zero.
struct Band6Args {
  const double* band;  // [11][7][n]
  double c[FQ_M6_TERMS];
  double sbeta;
  int n, ld;
};

__global__ void k_omega_band6(Band6Args a, double* __restrict__ ore, double* __restrict__ oim) {
  const int total = 7 * a.ld;
  const size_t el = (size_t)7 * a.n;  // stride between basis elements
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
    const int d = q / a.ld, i = q % a.ld;
    double sr = 0.0, si = 0.0;
    if (i < a.n) {
      const double* b = a.band + (size_t)d * a.n + i;
      sr = a.c[0] * b[0];
      sr = fma(a.c[1], b[el], sr);
      sr = fma(a.c[3], b[3 * el], sr);
      sr = fma(a.c[4], b[4 * el], sr);
      sr = fma(a.c[9], b[9 * el], sr);
      sr = fma(a.c[10], b[10 * el], sr);
      si = a.c[2] * b[2 * el];
      si = fma(a.c[5], b[5 * el], si);
      si = fma(a.c[6], b[6 * el], si);
      si = fma(a.c[7], b[7 * el], si);
      si = fma(a.c[8], b[8 * el], si);
      if (d == 3) sr -= a.sbeta;
    }
    ore[q] = sr;
    oim[q] = si;
  }
}

// One Chebyshev term with a heptadiagonal Omega~ (Eq. 10), FP64, streaming as k_term_tri: four
// entries of one state per thread, y_i = sum_{d = -3..3} Omega~[i][i + d] x_{i + d}.
__global__ void __launch_bounds__(256)
k_term_band6(const double* __restrict__ ore, const double* __restrict__ oim, int ld, const double* __restrict__ cur_re,
             const double* __restrict__ cur_im, const double* prev_re, const double* prev_im, double* acc_re,
             double* acc_im, double* out_re, double* out_im, fq_term t) {
  const int j = blockIdx.y;
  const int i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (i0 >= ld) return;
  const size_t row = (size_t)j * ld;
  double xr[10], xi[10];  // x_{i0 - 3} .. x_{i0 + 6}
#pragma unroll
  for (int u = 0; u < 10; ++u) {
    const int k = i0 - 3 + u;
    const bool in = k >= 0 && k < ld;
    xr[u] = in ? cur_re[row + k] : 0.0;
    xi[u] = in ? cur_im[row + k] : 0.0;
  }
  double pr[4], pi[4], ar[4], ai[4];
  if (!t.first) {
    Quad<double>::load(prev_re + row + i0, pr);
    Quad<double>::load(prev_im + row + i0, pi);
    Quad<double>::load(acc_re + row + i0, ar);
    Quad<double>::load(acc_im + row + i0, ai);
  }
  double o_r[4], o_i[4], a_r[4], a_i[4];
  bool bad = false;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    double yr = 0.0, yi = 0.0;
#pragma unroll
    for (int d = 0; d < 7; ++d) {
      const double wr = ore[(size_t)d * ld + i0 + q], wi = oim[(size_t)d * ld + i0 + q];
      yr = fma(wr, xr[q + d], fma(-wi, xi[q + d], yr));
      yi = fma(wr, xi[q + d], fma(wi, xr[q + d], yi));
    }
    double nr, ni, sr, si;
    if (t.first) {
      nr = yi;
      ni = -yr;
      sr = t.coef0 * xr[q + 3] + t.coef * nr;
      si = t.coef0 * xi[q + 3] + t.coef * ni;
    } else {
      nr = 2.0 * yi + pr[q];
      ni = -2.0 * yr + pi[q];
      sr = ar[q] + t.coef * nr;
      si = ai[q] + t.coef * ni;
    }
    bad |= !(nr * nr + ni * ni <= t.bound2);
    if (t.last) {
      o_r[q] = t.ph_re * sr - t.ph_im * si;
      o_i[q] = t.ph_re * si + t.ph_im * sr;
    } else {
      o_r[q] = nr;
      o_i[q] = ni;
      a_r[q] = sr;
      a_i[q] = si;
    }
  }
  if (bad) atomicOr(t.status, FQ_BIT_BOUND);
  Quad<double>::store(out_re + row + i0, o_r);
  Quad<double>::store(out_im + row + i0, o_i);
  if (!t.last) {
    Quad<double>::store(acc_re + row + i0, a_r);
    Quad<double>::store(acc_im + row + i0, a_i);
  }
}

// ------------------------------------------------------------------ unitarity defect
// D[c][j] = sum_i conj(U[i][c]) U[i][j] - delta_cj for up to 16 listed columns c (chunk
// blockIdx.y) and the 256 columns j of this block: U is streamed once per chunk, row by row,
// with the chunk's 16 entries of the row staged in shared memory.  Per block: the largest |D|
// and the sum of |D|^2.
__global__ void __launch_bounds__(256) k_defect(const double2* __restrict__ u, int n, const int32_t* __restrict__ cols,
                                                int k, double* partial) {
  constexpr int KC = 16;
  __shared__ double2 srow[KC];
  __shared__ int scol[KC];
  __shared__ double smx[256], sss[256];
  const int c0 = blockIdx.y * KC;
  const int kc = min(KC, k - c0);
  if (threadIdx.x < KC) {
    int r = c0 + threadIdx.x;
    scol[threadIdx.x] = threadIdx.x < kc ? (cols ? cols[r] : r) : -1;
  }
  __syncthreads();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  double sr[KC], si[KC];
#pragma unroll
  for (int q = 0; q < KC; ++q) sr[q] = si[q] = 0.0;
  for (int i = 0; i < n; ++i) {
    if (threadIdx.x < KC) {
      int c = scol[threadIdx.x];
      srow[threadIdx.x] = (c >= 0 && c < n) ? u[(size_t)i * n + c] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    double2 b = j < n ? u[(size_t)i * n + j] : make_double2(0.0, 0.0);
#pragma unroll
    for (int q = 0; q < KC; ++q) {
      double2 a = srow[q];
      sr[q] = fma(a.x, b.x, fma(a.y, b.y, sr[q]));
      si[q] = fma(a.x, b.y, fma(-a.y, b.x, si[q]));
    }
    __syncthreads();
  }
  double mx = 0.0, ss = 0.0;
  if (j < n) {
#pragma unroll
    for (int q = 0; q < KC; ++q) {
      if (q < kc) {
        double r = sr[q] - (scol[q] == j ? 1.0 : 0.0);
        double a2 = r * r + si[q] * si[q];
        mx = fmax(mx, sqrt(a2));
        ss += a2;
      }
    }
  }
  smx[threadIdx.x] = mx;
  sss[threadIdx.x] = ss;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      smx[threadIdx.x] = fmax(smx[threadIdx.x], smx[threadIdx.x + w]);
      sss[threadIdx.x] += sss[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[2 * ((size_t)blockIdx.y * gridDim.x + blockIdx.x)] = smx[0];
    partial[2 * ((size_t)blockIdx.y * gridDim.x + blockIdx.x) + 1] = sss[0];
  }
}

int grid_for(size_t total, int threads) {
  size_t b = (total + threads - 1) / threads;
  if (b > 152 * 64) b = 152 * 64;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

// ------------------------------------------------------------------ launchers
void fq_launch_load_states(const double* x, fq_blk<double> out, int nc, int n, int ld, cudaStream_t s) {
  k_load_states<double><<<grid_for((size_t)nc * ld, 256), 256, 0, s>>>((const double2*)x, out.re, out.im, nc, n, ld);
}
void fq_launch_load_states_f32(const double* x, fq_blk<float> out, int nc, int n, int ld, cudaStream_t s) {
  k_load_states<float><<<grid_for((size_t)nc * ld, 256), 256, 0, s>>>((const double2*)x, out.re, out.im, nc, n, ld);
}
void fq_launch_basis_rows(double* x, int nc, int n, int j0, cudaStream_t s) {
  k_basis_rows<<<grid_for((size_t)nc * n, 256), 256, 0, s>>>((double2*)x, nc, n, j0);
}
void fq_launch_identity_f64(fq_blk<double> out, int nc, int n, int ld, cudaStream_t s) {
  k_identity<double><<<grid_for((size_t)nc * ld, 256), 256, 0, s>>>(out.re, out.im, nc, n, ld);
}
void fq_launch_identity_f32(fq_blk<float> out, int nc, int n, int ld, cudaStream_t s) {
  k_identity<float><<<grid_for((size_t)nc * ld, 256), 256, 0, s>>>(out.re, out.im, nc, n, ld);
}
void fq_launch_store_states_f64(fq_blk<double> in, double* x, int nc, int n, int ld, cudaStream_t s) {
  k_store_states<double><<<grid_for((size_t)nc * n, 256), 256, 0, s>>>(in.re, in.im, (double2*)x, nc, n, ld);
}
void fq_launch_store_states_f32(fq_blk<float> in, double* x, int nc, int n, int ld, cudaStream_t s) {
  k_store_states<float><<<grid_for((size_t)nc * n, 256), 256, 0, s>>>(in.re, in.im, (double2*)x, nc, n, ld);
}
void fq_launch_store_transpose_f64(fq_blk<double> in, double* u, int n, int ld, cudaStream_t s) {
  dim3 g((n + 31) / 32, (n + 31) / 32), b(32, 8);
  k_store_transpose<double><<<g, b, 0, s>>>(in.re, in.im, (double2*)u, n, ld);
}
void fq_launch_store_transpose_f32(fq_blk<float> in, double* u, int n, int ld, cudaStream_t s) {
  dim3 g((n + 31) / 32, (n + 31) / 32), b(32, 8);
  k_store_transpose<float><<<g, b, 0, s>>>(in.re, in.im, (double2*)u, n, ld);
}

void fq_launch_gemm_f64(const double* a, const double* b, double* c, int n, double alpha, double beta, cudaStream_t s) {
  dim3 g((n + 15) / 16, (n + 15) / 16), blk(16, 16);
  k_gemm_f64<<<g, blk, 0, s>>>(a, b, c, n, alpha, beta);
}

void fq_launch_omega_dense_f64(const double* h0, const double* h1, const double* k, int n, double sa, double sb,
                               double sc, double sbeta, double* S, double* A, cudaStream_t s) {
  k_omega_dense_f64<<<grid_for((size_t)n * n, 256), 256, 0, s>>>(h0, h1, k, n, sa, sb, sc, sbeta, S, A);
}

Omega6Args omega6_args(const fq_plan* p, const double* c) {
  Omega6Args a;
  const size_t nn = (size_t)p->n * p->n;
  a.m[0] = p->d_h0;
  a.m[1] = p->d_h1;
  a.m[2] = p->d_k;
  for (int q = 0; q < 8; ++q) a.m[3 + q] = p->d_cm + q * nn;
  for (int q = 0; q < FQ_M6_TERMS; ++q) a.c[q] = c[q];
  a.sbeta = p->sbeta;
  a.n = p->n;
  return a;
}

void fq_launch_omega6_f64(const fq_plan* p, const double* c, double* S, double* A, cudaStream_t s) {
  k_omega6_f64<<<grid_for((size_t)p->n * p->n, 256), 256, 0, s>>>(omega6_args(p, c), S, A);
}

void fq_launch_frobenius(const double* a, size_t count, double* out, cudaStream_t s) {
  k_frobenius<<<grid_for(count, 256), 256, 0, s>>>(a, count, out);
}

void fq_launch_term_dense_f64(const double* S, const double* A, int n, fq_blk<double> cur, fq_blk<double> prev,
                              fq_blk<double> acc, fq_blk<double> out, int nc, const fq_term& t, cudaStream_t s) {
  // Smaller tiles when the grid would leave most of the 152 SMs idle (FP64 is ALU-bound).
  const long big = (long)((n + 31) / 32) * ((nc + 31) / 32);
  if (big >= 2 * 152) {
    dim3 g((n + 31) / 32, (nc + 31) / 32);
    if (A)
      k_term_dense_f64<32, 32, 16, 2, 2, true><<<g, 256, 0, s>>>(S, A, n, cur.re, cur.im, prev.re, prev.im, acc.re,
                                                                 acc.im, out.re, out.im, nc, t);
    else
      k_term_dense_f64<32, 32, 16, 2, 2, false><<<g, 256, 0, s>>>(S, A, n, cur.re, cur.im, prev.re, prev.im, acc.re,
                                                                  acc.im, out.re, out.im, nc, t);
  } else {
    dim3 g((n + 7) / 8, (nc + 7) / 8);
    if (A)
      k_term_dense_f64<8, 8, 32, 1, 1, true><<<g, 64, 0, s>>>(S, A, n, cur.re, cur.im, prev.re, prev.im, acc.re,
                                                              acc.im, out.re, out.im, nc, t);
    else
      k_term_dense_f64<8, 8, 32, 1, 1, false><<<g, 64, 0, s>>>(S, A, n, cur.re, cur.im, prev.re, prev.im, acc.re,
                                                               acc.im, out.re, out.im, nc, t);
  }
}

void fq_launch_tri_coeffs_f64(const fq_plan* p, int m_begin, int nsteps, double scale, double* d, double* er,
                              double* ei, cudaStream_t s) {
  const int ld = (p->n + 3) & ~3;
  k_tri_coeffs<double><<<grid_for((size_t)nsteps * ld, 256), 256, 0, s>>>(
      p->d_h0, p->d_h0o, p->d_h1, p->d_k, p->d_scal, p->n, ld, p->steps, m_begin, nsteps, p->sbeta, scale, d, er, ei);
}
void fq_launch_tri_coeffs_f32(const fq_plan* p, int m_begin, int nsteps, double scale, float* d, float* er,
                              float* ei, cudaStream_t s) {
  const int ld = (p->n + 3) & ~3;
  k_tri_coeffs<float><<<grid_for((size_t)nsteps * ld, 256), 256, 0, s>>>(
      p->d_h0, p->d_h0o, p->d_h1, p->d_k, p->d_scal, p->n, ld, p->steps, m_begin, nsteps, p->sbeta, scale, d, er, ei);
}

void fq_launch_omega_band6(const fq_plan* p, const double* c, double* ore, double* oim, int ld, cudaStream_t s) {
  Band6Args a;
  a.band = p->d_cm;
  for (int q = 0; q < FQ_M6_TERMS; ++q) a.c[q] = c[q];
  a.sbeta = p->sbeta;
  a.n = p->n;
  a.ld = ld;
  k_omega_band6<<<grid_for((size_t)7 * ld, 256), 256, 0, s>>>(a, ore, oim);
}

void fq_launch_term_band6_f64(const double* ore, const double* oim, int n, fq_blk<double> cur, fq_blk<double> prev,
                              fq_blk<double> acc, fq_blk<double> out, int nc, int ld, const fq_term& t,
                              cudaStream_t s) {
  (void)n;
  for (int r0 = 0; r0 < nc; r0 += 65535) {  // gridDim.y limit
    const int rows = nc - r0 < 65535 ? nc - r0 : 65535;
    const size_t o = (size_t)r0 * ld;
    dim3 g((ld / 4 + 255) / 256, rows);
    k_term_band6<<<g, 256, 0, s>>>(ore, oim, ld, cur.re + o, cur.im + o, prev.re + o, prev.im + o, acc.re + o,
                                   acc.im + o, out.re + o, out.im + o, t);
  }
}

void fq_launch_term_tri_f64(const double* d, const double* er, const double* ei, int n, fq_blk<double> cur,
                            fq_blk<double> prev, fq_blk<double> acc, fq_blk<double> out, int nc, int ld,
                            const fq_term& t, cudaStream_t s) {
  (void)n;
  for (int r0 = 0; r0 < nc; r0 += 65535) {  // gridDim.y limit
    const int rows = nc - r0 < 65535 ? nc - r0 : 65535;
    const size_t o = (size_t)r0 * ld;
    dim3 g((ld / 4 + 255) / 256, rows);
    k_term_tri<double><<<g, 256, 0, s>>>(d, er, ei, ld, cur.re + o, cur.im + o, prev.re + o, prev.im + o, acc.re + o,
                                         acc.im + o, out.re + o, out.im + o, t);
  }
}
void fq_launch_term_tri_f32(const float* d, const float* er, const float* ei, int n, fq_blk<float> cur,
                            fq_blk<float> prev, fq_blk<float> acc, fq_blk<float> out, int nc, int ld,
                            const fq_term& t, cudaStream_t s) {
  (void)n;
  for (int r0 = 0; r0 < nc; r0 += 65535) {  // gridDim.y limit
    const int rows = nc - r0 < 65535 ? nc - r0 : 65535;
    const size_t o = (size_t)r0 * ld;
    dim3 g((ld / 4 + 255) / 256, rows);
    k_term_tri<float><<<g, 256, 0, s>>>(d, er, ei, ld, cur.re + o, cur.im + o, prev.re + o, prev.im + o, acc.re + o,
                                        acc.im + o, out.re + o, out.im + o, t);
  }
}

namespace {
// y = (h0 + g h1) x (which 0), h0 x (1) or h1 x (2): dense row-major FP64, one warp per row
// (the Lanczos matrix-vector products of the spectral bounds, stage a1)
__global__ void k_symv2(const double* __restrict__ h0, const double* __restrict__ h1, double g, int which,
                        const double* __restrict__ x, double* __restrict__ y, int n) {
  const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= n) return;
  const double* a = h0 + (size_t)row * n;
  const double* b = h1 + (size_t)row * n;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) {
    const double xv = x[j];
    if (which == 0) s = fma(fma(g, b[j], a[j]), xv, s);
    else if (which == 1) s = fma(a[j], xv, s);
    else s = fma(b[j], xv, s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) y[row] = s;
}

}  // namespace

void fq_launch_symv2(const double* h0, const double* h1, double g, int which, const double* x, double* y, int n,
                     cudaStream_t s) {
  k_symv2<<<(n + 7) / 8, 256, 0, s>>>(h0, h1, g, which, x, y, n);
}

namespace {
// Bounded wait on an mbarrier nobody arrives on (the same try_wait loop as the pipelines'), then
// the timeout bit: the diagnostic of floquet_selftest_wait.
__global__ void k_wait_probe(unsigned int* status, long long cycles) {
  __shared__ __align__(8) unsigned long long bar;
  const unsigned addr = (unsigned)__cvta_generic_to_shared(&bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(1) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  const long long t0 = clock64();
  bool done = false;
  while (!done && clock64() - t0 < cycles) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(addr), "r"(0)
        : "memory");
    done = ok != 0;
  }
  if (!done) atomicOr(status, FQ_BIT_TIMEOUT);
}
}  // namespace

void fq_launch_wait_probe(unsigned int* status, long long cycles, cudaStream_t s) {
  k_wait_probe<<<1, 1, 0, s>>>(status, cycles);
}

namespace {
// FP32 rate probe: each thread runs independent chains of `iters` fused multiply-adds, 8 chains
// packed over lane pairs (FFMA2) or 16 scalar chains, and writes their sum so no work is dropped.
template <bool PACKED>
__global__ void __launch_bounds__(256) k_fp32_probe(float* out, int iters, float a, float b) {
  const float s0 = 1e-3f * (float)(threadIdx.x & 31);
  float t = 0.f;
  if (PACKED) {
    float2 acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = make_float2(s0 + k, s0 - k);
    const float2 A = make_float2(a, a), B = make_float2(b, b);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k] = __ffma2_rn(acc[k], A, B);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) t += acc[k].x + acc[k].y;
  } else {
    float acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = s0 + k;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int k = 0; k < 16; ++k) acc[k] = fmaf(acc[k], a, b);
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) t += acc[k];
  }
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = t;
}
}  // namespace

double fq_launch_fp32_probe(int packed, int iters, float* out, int blocks, cudaStream_t s) {
  if (packed) k_fp32_probe<true><<<blocks, 256, 0, s>>>(out, iters, 0.999f, 1e-3f);
  else k_fp32_probe<false><<<blocks, 256, 0, s>>>(out, iters, 0.999f, 1e-3f);
  return (double)blocks * 256 * iters * 16 * 2;  // 16 multiply-adds of 2 flop per thread and iteration
}

void fq_launch_defect(const double* u, int n, const int32_t* cols, int k, double* partial, cudaStream_t s) {
  dim3 g((n + 255) / 256, (k + 15) / 16);
  k_defect<<<g, 256, 0, s>>>((const double2*)u, n, cols, k, partial);
}
