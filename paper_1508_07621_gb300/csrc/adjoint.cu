// floquet_grad: gate-fidelity loss L = 1 - |Tr(W^+ U_T)|^2 / N^2 and dL/df_m for piecewise-constant
// amplitudes f_m, by reverse mode through the Magnus-Chebyshev chain (Eqs. 9, 10, 12), FP64.
//
// Piecewise-constant f makes f' = f'' = 0 inside a step, so Omega_m = h (H0 + f_m H1) (Eq. 14) and,
// with bounds frozen by the plan, Omega~_m = (H0 + f_m H1 - beta)/Delta E is REAL symmetric and
// dOmega~_m/df_m = E = H1/Delta E.  With G_m = dL/dconj(X_m) (convention dL = 2 Re <G, dX>,
// <A, B> = Tr(A^+ B)), step m's adjoint is the Clenshaw-form recurrence
//   bbar_l = conj(e^{-i beta h}) a_l G_m + conj(w_{l+1}) Omega~ bbar_{l+1} + bbar_{l+2}
//   (bbar_{L+1} = bbar_{L+2} = 0, w_1 = -i, w_l = -2i for l >= 2),
//   G_{m-1} = bbar_0 = U_m^+ G_m,   dL/df_m = 2 Re sum_{l=1}^{L} w_l <bbar_l, E psi_{l-1}>,
// where psi_l are step m's forward Chebyshev vectors.  Seed: G_M = -tau W / N^2, tau = Tr(W^+ U_T).
//
// Memory: X_m is kept every s = checkpoint_stride steps; each segment is recomputed forward once,
// keeping its psi_l, and then walked backward.  All matrices are stored as rows (row r = column r
// of the column-state matrix), so every product is the dense FP64 tile Y^T = X^T Omega~^T.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "dense_core.cuh"
#include "internal.h"

namespace {

constexpr int BJ = 32, BI = 32, BK = 16, TJ = 2, TI = 2, NTH = 256;

int grid_n(size_t total) {
  size_t b = (total + 255) / 256;
  return (int)std::min<size_t>(std::max<size_t>(b, 1), 152 * 64);
}

// S = (H0 + f_m H1) / Delta E - (beta / Delta E) 1   (f_m read from device memory)
__global__ void k_omega_pw(const double* __restrict__ h0, const double* __restrict__ h1, int n,
                           const double* __restrict__ f, int m, double inv_de, double sbeta, double* S) {
  const double fm = f[m];
  size_t total = (size_t)n * n;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(q / n), j = (int)(q % n);
    S[q] = (h0[q] + fm * h1[q]) * inv_de - (i == j ? sbeta : 0.0);
  }
}

__global__ void k_scale(const double* __restrict__ a, size_t total, double s, double* out) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x)
    out[q] = s * a[q];
}

__global__ void k_copy2(const double* __restrict__ ar, const double* __restrict__ ai, size_t total, double* br,
                        double* bi) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    br[q] = ar[q];
    bi[q] = ai[q];
  }
}

__global__ void k_identity_rows(double* re, double* im, int n) {
  size_t total = (size_t)n * n;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    re[q] = (q / n == q % n) ? 1.0 : 0.0;
    im[q] = 0.0;
  }
}

// bbar_L = cpa G  (cpa = conj(phase) a_L), elementwise
__global__ void k_scale_c(const double* __restrict__ gr, const double* __restrict__ gi, size_t total, double cr,
                          double ci, double* outr, double* outi) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const double a = gr[q], b = gi[q];
    outr[q] = cr * a - ci * b;
    outi[q] = cr * b + ci * a;
  }
}

// Adjoint term: out = cpa G + i cw (Omega~ b1) + b2   (b2 may be absent; out may alias b2)
__global__ void __launch_bounds__(NTH)
k_adj_term(const double* __restrict__ S, int n, const double* __restrict__ b1r, const double* __restrict__ b1i,
           const double* b2r, const double* b2i, const double* __restrict__ gr, const double* __restrict__ gi,
           double* outr, double* outi, double cpr, double cpi, double cw) {
  constexpr int NTX = BI / TI;
  const int tx = threadIdx.x % NTX, ty = threadIdx.x / NTX;
  const int j0 = blockIdx.y * BJ, i0 = blockIdx.x * BI;
  double yr[TJ][TI], yi[TJ][TI];
  dense_tile_f64<BJ, BI, BK, TJ, TI, false>(S, nullptr, n, b1r, b1i, n, j0, i0, yr, yi);
#pragma unroll
  for (int u = 0; u < TJ; ++u)
#pragma unroll
    for (int v = 0; v < TI; ++v) {
      const int j = j0 + ty * TJ + u, i = i0 + tx * TI + v;
      if (j < n && i < n) {
        const size_t idx = (size_t)j * n + i;
        const double g0 = gr[idx], g1 = gi[idx];
        double o_r = cpr * g0 - cpi * g1 - cw * yi[u][v];
        double o_i = cpr * g1 + cpi * g0 + cw * yr[u][v];
        if (b2r) {
          o_r += b2r[idx];
          o_i += b2i[idx];
        }
        outr[idx] = o_r;
        outi[idx] = o_i;
      }
    }
}

// partial[cta] = sum over the tile of conj(B[j][i]) (Psi E)[j][i]   (E real symmetric)
__global__ void __launch_bounds__(NTH)
k_dot(const double* __restrict__ E, int n, const double* __restrict__ pr, const double* __restrict__ pi,
      const double* __restrict__ br, const double* __restrict__ bi, double2* partial) {
  constexpr int NTX = BI / TI;
  const int tx = threadIdx.x % NTX, ty = threadIdx.x / NTX;
  const int j0 = blockIdx.y * BJ, i0 = blockIdx.x * BI;
  double yr[TJ][TI], yi[TJ][TI];
  dense_tile_f64<BJ, BI, BK, TJ, TI, false>(E, nullptr, n, pr, pi, n, j0, i0, yr, yi);
  double sr = 0.0, si = 0.0;
#pragma unroll
  for (int u = 0; u < TJ; ++u)
#pragma unroll
    for (int v = 0; v < TI; ++v) {
      const int j = j0 + ty * TJ + u, i = i0 + tx * TI + v;
      if (j < n && i < n) {
        const size_t idx = (size_t)j * n + i;
        const double a = br[idx], b = bi[idx];
        sr += a * yr[u][v] + b * yi[u][v];
        si += a * yi[u][v] - b * yr[u][v];
      }
    }
  __shared__ double rr[NTH], ri[NTH];
  rr[threadIdx.x] = sr;
  ri[threadIdx.x] = si;
  __syncthreads();
  for (int w = NTH / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      rr[threadIdx.x] += rr[threadIdx.x + w];
      ri[threadIdx.x] += ri[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = make_double2(rr[0], ri[0]);
}

// tau partials: sum over rows j of X_M^T (states) of conj(W[i][j]) X^T[j][i]
__global__ void k_trace_partials(const double2* __restrict__ W, const double* __restrict__ xr,
                                 const double* __restrict__ xi, int n, double2* partial) {
  const int j = blockIdx.x;  // state row = column j of U_T
  double sr = 0.0, si = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double2 w = W[(size_t)i * n + j];
    const double a = xr[(size_t)j * n + i], b = xi[(size_t)j * n + i];
    sr += w.x * a + w.y * b;
    si += w.x * b - w.y * a;
  }
  __shared__ double rr[256], ri[256];
  rr[threadIdx.x] = sr;
  ri[threadIdx.x] = si;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      rr[threadIdx.x] += rr[threadIdx.x + w];
      ri[threadIdx.x] += ri[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[j] = make_double2(rr[0], ri[0]);
}

// one CTA: tau = sum partials; loss = 1 - |tau|^2 / N^2
__global__ void k_loss(const double2* __restrict__ partial, int count, int n, double* loss, double2* tau) {
  __shared__ double rr[256], ri[256];
  double sr = 0.0, si = 0.0;
  for (int q = threadIdx.x; q < count; q += blockDim.x) {
    sr += partial[q].x;
    si += partial[q].y;
  }
  rr[threadIdx.x] = sr;
  ri[threadIdx.x] = si;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      rr[threadIdx.x] += rr[threadIdx.x + w];
      ri[threadIdx.x] += ri[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double nn = (double)n * n;
    *tau = make_double2(rr[0], ri[0]);
    *loss = 1.0 - (rr[0] * rr[0] + ri[0] * ri[0]) / nn;
  }
}

// seed G_M = -tau W / N^2, stored as rows: G^T[j][i] = G[i][j]
__global__ void k_seed(const double2* __restrict__ W, const double2* __restrict__ tau, int n, double* gr,
                       double* gi) {
  const double2 t = *tau;
  const double s = -1.0 / ((double)n * n);
  size_t total = (size_t)n * n;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(q / n), i = (int)(q % n);
    const double2 w = W[(size_t)i * n + j];
    gr[q] = s * (t.x * w.x - t.y * w.y);
    gi[q] = s * (t.x * w.y + t.y * w.x);
  }
}

// grad[m] = 2 Re sum_{l=1}^{L} w_l D_l, D_l = sum of partials of l; w_1 = -i, w_l = -2i:
// Re(-i c D) = c Im(D).
__global__ void k_grad_reduce(const double2* __restrict__ partial, int ncta, int L, double* grad_m) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int l = 1; l <= L; ++l) {
    const double c = l == 1 ? 1.0 : 2.0;
    for (int q = threadIdx.x; q < ncta; q += blockDim.x) acc += c * partial[(size_t)l * ncta + q].y;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *grad_m = 2.0 * red[0];
}

struct Mat {
  double* re;
  double* im;
};

struct GradWs {
  double* S;
  double* E;
  Mat acc, x[3], ck_base, slot_base, b[3];
  size_t nn;
  int nseg, nslots;
  double2* partial;
  double2* tau_partial;
  double2* tau;
  Mat ck(int k) const { return Mat{ck_base.re + 2 * nn * (size_t)k, ck_base.re + 2 * nn * (size_t)k + nn}; }
  Mat slot(int q) const { return Mat{slot_base.re + 2 * nn * (size_t)q, slot_base.re + 2 * nn * (size_t)q + nn}; }
};

size_t up(size_t x) { return (x + 255) & ~(size_t)255; }

size_t grad_layout(const fq_plan* p, void* base, GradWs* w) {
  const size_t n = p->n, nn = n * n;
  const int s = p->stride, M = p->steps, L = p->L;
  const int nseg = (M + s - 1) / s;
  const int nslots = s * L + 1;
  const size_t ncta = ((n + BI - 1) / BI) * ((n + BJ - 1) / BJ);
  char* b = (char*)base;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* q = b ? b + off : nullptr;
    off += up(bytes);
    return q;
  };
  GradWs g{};
  g.nn = nn;
  g.nseg = nseg;
  g.nslots = nslots;
  g.S = (double*)take(nn * 8);
  g.E = (double*)take(nn * 8);
  auto mat = [&]() {
    double* r = (double*)take(2 * nn * 8);
    return Mat{r, r ? r + nn : nullptr};
  };
  g.acc = mat();
  for (int q = 0; q < 3; ++q) g.x[q] = mat();
  for (int q = 0; q < 3; ++q) g.b[q] = mat();
  double* ck = (double*)take(2 * nn * 8 * (size_t)nseg);
  g.ck_base = Mat{ck, nullptr};
  double* sl = (double*)take(2 * nn * 8 * (size_t)nslots);
  g.slot_base = Mat{sl, nullptr};
  g.partial = (double2*)take(sizeof(double2) * (L + 1) * ncta);
  g.tau_partial = (double2*)take(sizeof(double2) * n);
  g.tau = (double2*)take(sizeof(double2));
  if (w) *w = g;
  return off;
}

// One forward step m on rows: X_{m-1} (in `in`) -> X_m (in `out`).  With `psi`, psi_1..psi_{L-1}
// go to psi[1..L-1] (kept for the backward pass); without, psi_1 and psi_2 go to tmp0 / tmp1
// and later psi_{l+1} overwrite psi_{l-1} in place.  `in` is only read elementwise after the
// first product, so tmp1 may be `in` itself when `in` is scratch; it must differ when `in` is
// a checkpoint.
void forward_step(const fq_plan* p, const GradWs& w, const double* d_f, int m, Mat in, Mat out, const Mat* psi,
                  Mat tmp0, Mat tmp1, cudaStream_t s) {
  const int n = p->n, L = p->L;
  k_omega_pw<<<grid_n(w.nn), 256, 0, s>>>(p->d_h0, p->d_h1, n, d_f, m, 1.0 / p->delta_e, p->sbeta, w.S);
  fq_term t{};
  t.coef0 = p->cheb[0];
  t.ph_re = p->phase_re;
  t.ph_im = p->phase_im;
  t.bound2 = 1.0 + 1e-9;
  t.status = p->d_status;
  // psi_0 = in; psi_{l+1} goes to psi[l+1] (kept) or alternates tmp0 / tmp1 / in-place
  Mat cur = in, prev = in;
  Mat bufs[2] = {tmp0, tmp1};
  for (int l = 0; l < L; ++l) {
    t.first = l == 0;
    t.last = l == L - 1;
    t.coef = p->cheb[l + 1];
    Mat o;
    if (t.last) o = out;
    else if (psi) o = psi[l + 1];
    else o = l == 0 ? bufs[0] : (l == 1 ? bufs[1] : prev);  // in place over psi_{l-1} when not kept
    fq_launch_term_dense_f64(w.S, nullptr, n, fq_blk<double>{cur.re, cur.im}, fq_blk<double>{prev.re, prev.im},
                             fq_blk<double>{w.acc.re, w.acc.im}, fq_blk<double>{o.re, o.im}, n, t, s);
    prev = cur;
    cur = o;
  }
}

}  // namespace

void fq_launch_loss(const double2* partial, int count, int n, double* loss, double2* tau, cudaStream_t s) {
  k_loss<<<1, 256, 0, s>>>(partial, count, n, loss, tau);
}

void fq_launch_grad_reduce(const double2* partial, int ncta, int L, double* grad_m, cudaStream_t s) {
  k_grad_reduce<<<1, 256, 0, s>>>(partial, ncta, L, grad_m);
}

void fq_launch_trace_f64(const double* W, const double* xr, const double* xi, int n, double2* partial,
                         cudaStream_t s) {
  k_trace_partials<<<n, 256, 0, s>>>((const double2*)W, xr, xi, n, partial);
}

void fq_launch_seed_f64(const double* W, const double2* tau, int n, double* gr, double* gi, cudaStream_t s) {
  k_seed<<<grid_n((size_t)n * n), 256, 0, s>>>((const double2*)W, tau, n, gr, gi);
}

extern "C" size_t floquet_grad_workspace_size(const fq_plan* p) {
  if (!p || p->format != FQ_DENSE || p->drive_kind != FQ_DRIVE_PIECEWISE) return 0;
  if (p->precision == FQ_BF16X3 || p->precision == FQ_BF16X6) return fq_grad_split_workspace(p);
  if (p->precision == FQ_OZAKI) return fq_grad_ozaki_workspace(p);
  return grad_layout(p, nullptr, nullptr);
}

static fq_status floquet_grad_body(fq_plan* p, const double* d_f, const void* d_W, double* d_loss, double* d_grad,
                                   void* d_ws, size_t ws_bytes, void* stream) {
  if (!p || !d_f || !d_W || !d_loss || !d_grad) {
    fq_set_error("floquet_grad: NULL argument");
    return FQ_EINVAL;
  }
  if (p->format != FQ_DENSE || p->drive_kind != FQ_DRIVE_PIECEWISE) {
    fq_set_error("floquet_grad needs a dense plan with FQ_DRIVE_PIECEWISE");
    return FQ_EINVAL;
  }
  if (p->precision != FQ_FP64 && p->precision != FQ_BF16X3 && p->precision != FQ_BF16X6 &&
      p->precision != FQ_OZAKI) {
    fq_set_error("floquet_grad: FQ_FP64, FQ_BF16X3, FQ_BF16X6 and FQ_OZAKI are built");
    return FQ_EUNSUPPORTED;
  }
  const size_t need = floquet_grad_workspace_size(p);
  if (!d_ws || ws_bytes < need || ((uintptr_t)d_ws & 255)) {
    fq_set_error("floquet_grad: workspace must be >= %zu bytes, 256-byte aligned (got %zu)", need, ws_bytes);
    return FQ_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (p->precision == FQ_OZAKI) return fq_grad_ozaki(p, d_f, d_W, d_loss, d_grad, d_ws, s);
  if (p->precision != FQ_FP64) return fq_grad_split(p, d_f, d_W, d_loss, d_grad, d_ws, s);
  GradWs w;
  grad_layout(p, d_ws, &w);
  const int n = p->n, M = p->steps, L = p->L, S = p->stride;
  const size_t nn = w.nn;
  const dim3 gg((n + BI - 1) / BI, (n + BJ - 1) / BJ);
  const int ncta = gg.x * gg.y;

  k_scale<<<grid_n(nn), 256, 0, s>>>(p->d_h1, nn, 1.0 / p->delta_e, w.E);
  // ---- forward sweep with checkpoints X_{kS}
  k_identity_rows<<<grid_n(nn), 256, 0, s>>>(w.ck(0).re, w.ck(0).im, n);
  Mat x = w.ck(0);
  int xi = 0;
  for (int m = 0; m < M; ++m) {
    Mat out = w.x[xi];
    forward_step(p, w, d_f, m, x, out, nullptr, w.x[(xi + 1) % 3], w.x[(xi + 2) % 3], s);
    x = out;
    xi = (xi + 1) % 3;
    if ((m + 1) % S == 0 && (m + 1) / S < w.nseg) {
      Mat c = w.ck((m + 1) / S);
      k_copy2<<<grid_n(nn), 256, 0, s>>>(x.re, x.im, nn, c.re, c.im);
      x = c;
    }
  }
  // ---- loss and seed
  k_trace_partials<<<n, 256, 0, s>>>((const double2*)d_W, x.re, x.im, n, w.tau_partial);
  k_loss<<<1, 256, 0, s>>>(w.tau_partial, n, n, d_loss, w.tau);
  Mat G = w.b[2], B0 = w.b[0], B1 = w.b[1];
  k_seed<<<grid_n(nn), 256, 0, s>>>((const double2*)d_W, w.tau, n, G.re, G.im);
  // ---- backward, one checkpoint segment at a time
  const double cph_r = p->phase_re, cph_i = -p->phase_im;  // conj(e^{-i beta h})
  for (int k = w.nseg - 1; k >= 0; --k) {
    const int m0 = k * S, m1 = std::min(M, m0 + S);
    // recompute the segment forward, keeping every psi_l (slot st*L + l; X_{m+1} at slot (st+1)*L)
    k_copy2<<<grid_n(nn), 256, 0, s>>>(w.ck(k).re, w.ck(k).im, nn, w.slot(0).re, w.slot(0).im);
    for (int st = 0; st < m1 - m0; ++st) {
      std::vector<Mat> psi(L + 1);
      for (int l = 0; l < L; ++l) psi[l] = w.slot(st * L + l);
      forward_step(p, w, d_f, m0 + st, psi[0], w.slot((st + 1) * L), psi.data(), Mat{}, Mat{}, s);
    }
    for (int st = m1 - m0 - 1; st >= 0; --st) {
      const int m = m0 + st;
      k_omega_pw<<<grid_n(nn), 256, 0, s>>>(p->d_h0, p->d_h1, n, d_f, m, 1.0 / p->delta_e, p->sbeta, w.S);
      // bbar_L = conj(phase) a_L G
      Mat bl1 = B0, bl2 = B1;  // bbar_{l+1}, bbar_{l+2}
      k_scale_c<<<grid_n(nn), 256, 0, s>>>(G.re, G.im, nn, cph_r * p->cheb[L], cph_i * p->cheb[L], bl1.re, bl1.im);
      Mat psiL1 = w.slot(st * L + L - 1);
      k_dot<<<gg, NTH, 0, s>>>(w.E, n, psiL1.re, psiL1.im, bl1.re, bl1.im, w.partial + (size_t)L * ncta);
      bool have2 = false;
      for (int l = L - 1; l >= 0; --l) {
        const double a = p->cheb[l];
        const double cw = l == 0 ? 1.0 : 2.0;
        // out (bbar_l) replaces bbar_{l+2}
        k_adj_term<<<gg, NTH, 0, s>>>(w.S, n, bl1.re, bl1.im, have2 ? bl2.re : nullptr, have2 ? bl2.im : nullptr,
                                      G.re, G.im, bl2.re, bl2.im, cph_r * a, cph_i * a, cw);
        if (l >= 1) {
          Mat ps = w.slot(st * L + l - 1);
          k_dot<<<gg, NTH, 0, s>>>(w.E, n, ps.re, ps.im, bl2.re, bl2.im, w.partial + (size_t)l * ncta);
        }
        std::swap(bl1, bl2);  // now bl1 = bbar_l, bl2 = bbar_{l+1}
        have2 = true;
      }
      k_grad_reduce<<<1, 256, 0, s>>>(w.partial, ncta, L, d_grad + m);
      // G_{m-1} = bbar_0 (in bl1); the old G buffer becomes scratch
      Mat old = G;
      G = bl1;
      B0 = bl2;
      B1 = old;
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fq_cuda_fail(e, "floquet_grad kernels");
  return FQ_OK;
}

extern "C" fq_status floquet_grad(fq_plan* p, const double* d_f, const void* d_W, double* d_loss, double* d_grad,
                                  void* d_ws, size_t ws_bytes, void* stream) {
  return fq_guard("floquet_grad", [&] {
    return floquet_grad_body(p, d_f, d_W, d_loss, d_grad, d_ws, ws_bytes, stream);
  });
}
