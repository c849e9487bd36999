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

// One Chebyshev term, dense FP64: Y^T[j][i] = sum_k Psi[j][k] (S[i][k] + i A[i][k]) followed by
// the fused epilogue.  BJ x BI output tile per CTA, (BJ/TJ) x (BI/TI) threads, TJ x TI
// complex outputs per thread, K staged through shared memory in BK slices.
template <int BJ, int BI, int BK, int TJ, int TI>
__global__ void __launch_bounds__((BJ / TJ) * (BI / TI))
k_term_dense_f64(const double* __restrict__ S, const double* __restrict__ A, int n,
                 const double* __restrict__ cur_re, const double* __restrict__ cur_im,
                 const double* prev_re, const double* prev_im, double* acc_re, double* acc_im,
                 double* out_re, double* out_im, int nc, fq_term t) {
  constexpr int NTX = BI / TI, NTY = BJ / TJ, NT = NTX * NTY;
  __shared__ double sPr[BK][BJ + 1], sPi[BK][BJ + 1], sS[BK][BI + 1], sA[BK][BI + 1];
  const int tx = threadIdx.x % NTX, ty = threadIdx.x / NTX;
  const int j0 = blockIdx.y * BJ, i0 = blockIdx.x * BI;
  double yr[TJ][TI], yi[TJ][TI];
#pragma unroll
  for (int a = 0; a < TJ; ++a)
#pragma unroll
    for (int b = 0; b < TI; ++b) yr[a][b] = yi[a][b] = 0.0;
  for (int k0 = 0; k0 < n; k0 += BK) {
    for (int q = threadIdx.x; q < BJ * BK; q += NT) {
      int r = q / BK, kk = q % BK, j = j0 + r, k = k0 + kk;
      bool ok = j < nc && k < n;
      sPr[kk][r] = ok ? cur_re[(size_t)j * n + k] : 0.0;
      sPi[kk][r] = ok ? cur_im[(size_t)j * n + k] : 0.0;
    }
    for (int q = threadIdx.x; q < BI * BK; q += NT) {
      int r = q / BK, kk = q % BK, i = i0 + r, k = k0 + kk;
      bool ok = i < n && k < n;
      sS[kk][r] = ok ? S[(size_t)i * n + k] : 0.0;
      sA[kk][r] = ok ? A[(size_t)i * n + k] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      double pr[TJ], pi[TJ], s[TI], a[TI];
#pragma unroll
      for (int q = 0; q < TJ; ++q) { pr[q] = sPr[kk][ty * TJ + q]; pi[q] = sPi[kk][ty * TJ + q]; }
#pragma unroll
      for (int q = 0; q < TI; ++q) { s[q] = sS[kk][tx * TI + q]; a[q] = sA[kk][tx * TI + q]; }
#pragma unroll
      for (int u = 0; u < TJ; ++u)
#pragma unroll
        for (int v = 0; v < TI; ++v) {
          yr[u][v] = fma(pr[u], s[v], fma(-pi[u], a[v], yr[u][v]));
          yi[u][v] = fma(pi[u], s[v], fma(pr[u], a[v], yi[u][v]));
        }
    }
    __syncthreads();
  }
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
// thread; rows are padded to ld (multiple of 4) with zeros.
template <typename T>
__global__ void __launch_bounds__(256)
k_term_tri(const T* __restrict__ d, const T* __restrict__ er, const T* __restrict__ ei, int ld,
           const T* __restrict__ cur_re, const T* __restrict__ cur_im, const T* prev_re, const T* prev_im,
           T* acc_re, T* acc_im, T* out_re, T* out_im, fq_term t) {
  const int j = blockIdx.y;
  const int i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (i0 >= ld) return;
  const size_t row = (size_t)j * ld;
  T cr[6], ci[6], dd[4], lr[5], li[5];
  cr[0] = i0 > 0 ? cur_re[row + i0 - 1] : (T)0;
  ci[0] = i0 > 0 ? cur_im[row + i0 - 1] : (T)0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    cr[q + 1] = cur_re[row + i0 + q];
    ci[q + 1] = cur_im[row + i0 + q];
    dd[q] = d[i0 + q];
    lr[q + 1] = er[i0 + q];
    li[q + 1] = ei[i0 + q];
  }
  cr[5] = i0 + 4 < ld ? cur_re[row + i0 + 4] : (T)0;
  ci[5] = i0 + 4 < ld ? cur_im[row + i0 + 4] : (T)0;
  lr[0] = i0 > 0 ? er[i0 - 1] : (T)0;
  li[0] = i0 > 0 ? ei[i0 - 1] : (T)0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    // y = d_i x_i + e_{i-1} x_{i-1} + conj(e_i) x_{i+1}
    T yr = dd[q] * cr[q + 1];
    T yi = dd[q] * ci[q + 1];
    yr = fma(lr[q], cr[q], fma(-li[q], ci[q], yr));
    yi = fma(lr[q], ci[q], fma(li[q], cr[q], yi));
    yr = fma(lr[q + 1], cr[q + 2], fma(li[q + 1], ci[q + 2], yr));
    yi = fma(lr[q + 1], ci[q + 2], fma(-li[q + 1], cr[q + 2], yi));
    term_epilogue<T>(yr, yi, cr[q + 1], ci[q + 1], prev_re, prev_im, acc_re, acc_im, out_re, out_im,
                     row + i0 + q, t);
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

void fq_launch_term_dense_f64(const double* S, const double* A, int n, fq_blk<double> cur, fq_blk<double> prev,
                              fq_blk<double> acc, fq_blk<double> out, int nc, const fq_term& t, cudaStream_t s) {
  // Smaller tiles when the grid would leave most of the 152 SMs idle (FP64 is ALU-bound).
  const long big = (long)((n + 31) / 32) * ((nc + 31) / 32);
  if (big >= 2 * 152) {
    dim3 g((n + 31) / 32, (nc + 31) / 32);
    k_term_dense_f64<32, 32, 16, 2, 2><<<g, 256, 0, s>>>(S, A, n, cur.re, cur.im, prev.re, prev.im, acc.re, acc.im,
                                                          out.re, out.im, nc, t);
  } else {
    dim3 g((n + 7) / 8, (nc + 7) / 8);
    k_term_dense_f64<8, 8, 32, 1, 1><<<g, 64, 0, s>>>(S, A, n, cur.re, cur.im, prev.re, prev.im, acc.re, acc.im,
                                                       out.re, out.im, nc, t);
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

void fq_launch_term_tri_f64(const double* d, const double* er, const double* ei, int n, fq_blk<double> cur,
                            fq_blk<double> prev, fq_blk<double> acc, fq_blk<double> out, int nc, int ld,
                            const fq_term& t, cudaStream_t s) {
  (void)n;
  dim3 g((ld / 4 + 255) / 256, nc);
  k_term_tri<double><<<g, 256, 0, s>>>(d, er, ei, ld, cur.re, cur.im, prev.re, prev.im, acc.re, acc.im, out.re,
                                       out.im, t);
}
void fq_launch_term_tri_f32(const float* d, const float* er, const float* ei, int n, fq_blk<float> cur,
                            fq_blk<float> prev, fq_blk<float> acc, fq_blk<float> out, int nc, int ld,
                            const fq_term& t, cudaStream_t s) {
  (void)n;
  dim3 g((ld / 4 + 255) / 256, nc);
  k_term_tri<float><<<g, 256, 0, s>>>(d, er, ei, ld, cur.re, cur.im, prev.re, prev.im, acc.re, acc.im, out.re,
                                      out.im, t);
}

void fq_launch_defect(const double* u, int n, const int32_t* cols, int k, double* partial, cudaStream_t s) {
  dim3 g((n + 255) / 256, (k + 15) / 16);
  k_defect<<<g, 256, 0, s>>>((const double2*)u, n, cols, k, partial);
}
