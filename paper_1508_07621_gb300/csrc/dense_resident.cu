// Resident dense chain for small N (FP64): a cluster of C = ceil(N/32) CTAs carries one state
// through every step of a chunk of the period, with the state on chip the whole time.
//
// The per-term dense path launches one tiled GEMM per Chebyshev term; at N = 64 each of those
// launches keeps only a handful of SMs busy and the chain is 1400 dependent launches long
// (M = 200, L = 7).  Here the independence of the columns of U_T (Algorithm 1 propagates each
// initial state on its own) is used instead: one cluster per state, each CTA owning 32 rows of
// Omega~_m, so 64 states fill 128 SMs and the whole chunk is one launch.
//
// Per step m (Eqs. 10-12): Phi_0 = X_{m-1}, Phi_1 = -i Omega~ Phi_0,
// Phi_{l+1} = -2i Omega~ Phi_l + Phi_{l-1}, X_m = e^{-i beta h} sum_{l<=L} a_l Phi_l.
// Each CTA keeps the full state vector Phi_l (N complex values) in shared memory, twice
// (double-buffered); a thread pair (row i, k-group g) holds 8 entries of row i of S_m and A_m
// (Omega~_m = S_m + i A_m) in registers, and the KG threads of a row reduce their partial
// sums by shuffles.  The row's first thread advances the recurrence and the accumulator in
// registers and writes the new entry of Phi into every CTA of the cluster (distributed shared
// memory); one cluster barrier per product publishes the vector.
//
// Omega~_m for the chunk's steps is formed beforehand in HBM (it is L2-resident: 64 steps x
// 2 x N^2 doubles = 4 MB at N = 64) by one batched launch (order 4) or one launch per step
// (order 6).
//
// FQ_DF32 runs the same chain in double-float arithmetic (dfl.cuh) on the FP32 pipes, which
// GB300 runs at many times its FP64 rate: Omega~ is converted once per step to FP32 pairs, the
// state lives in shared memory as packed complex pairs, and the states in HBM stay FP64.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "dfl.cuh"
#include "internal.h"

namespace {

constexpr int DR_ROWS = 32;   // rows of Omega~ per CTA
constexpr int DR_KPT = 8;     // entries of a row per thread
constexpr int DR_MAXN = 128;
constexpr int DR_CHUNK = 64;  // steps per launch
constexpr int DR_MAXL = 128;

struct DrCoef {
  double a[DR_MAXL + 1];
};

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// stores (x, y) at the same shared-memory offset as `local` in cluster CTA `rank`
__device__ __forceinline__ void st_cluster_f64x2(const void* local, unsigned rank, double x, double y) {
  const unsigned la = (unsigned)__cvta_generic_to_shared(local);
  unsigned ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(la), "r"(rank));
  asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(ra), "d"(x), "d"(y) : "memory");
}

// S, A: [nsteps][n][n] (Omega~ of the chunk's steps); x: planar states [nc][n], updated in place.
template <int ROWS, int KG>
__global__ void __launch_bounds__(ROWS* KG)
    k_dense_resident(const double* __restrict__ S, const double* __restrict__ A, int n, int nsteps, int L, int C,
                     DrCoef cf, double ph_re, double ph_im, double bound2, double* xr, double* xi,
                     unsigned* status) {
  constexpr int NT = ROWS * KG;
  constexpr int NV = KG * DR_KPT;  // vector length held per buffer (>= n)
  __shared__ double2 phi[2][NV];
  const int t = threadIdx.x, rl = t / KG, g = t % KG;
  const unsigned rank = C > 1 ? cluster_rank() : 0u;
  const int j = blockIdx.x / C;  // the state this cluster carries
  const int i = (int)rank * ROWS + rl;
  const bool own = g == 0 && i < n;
  for (int q = t; q < 2 * NV; q += NT) {
    const int b = q / NV, k = q % NV;
    phi[b][k] = b == 0 && k < n ? make_double2(xr[(size_t)j * n + k], xi[(size_t)j * n + k]) : make_double2(0.0, 0.0);
  }
  __syncthreads();
  if (C > 1) cluster_sync_all();  // every CTA of the cluster is running before remote stores
  const size_t nn = (size_t)n * n;
  int buf = 0;
  bool bad = false;
  for (int m = 0; m < nsteps; ++m) {
    double s[DR_KPT], a[DR_KPT];
#pragma unroll
    for (int q = 0; q < DR_KPT; ++q) {
      const int k = g + KG * q;
      const bool ok = i < n && k < n;
      s[q] = ok ? S[m * nn + (size_t)i * n + k] : 0.0;
      a[q] = ok ? A[m * nn + (size_t)i * n + k] : 0.0;
    }
    double accr = 0.0, acci = 0.0, pvr = 0.0, pvi = 0.0;
    for (int l = 0; l < L; ++l) {
      double yr = 0.0, yi = 0.0;
#pragma unroll
      for (int q = 0; q < DR_KPT; ++q) {
        const double2 v = phi[buf][g + KG * q];
        yr = fma(s[q], v.x, fma(-a[q], v.y, yr));
        yi = fma(s[q], v.y, fma(a[q], v.x, yi));
      }
#pragma unroll
      for (int o = KG / 2; o > 0; o >>= 1) {
        yr += __shfl_xor_sync(0xffffffffu, yr, o);
        yi += __shfl_xor_sync(0xffffffffu, yi, o);
      }
      if (own) {
        const double2 cur = phi[buf][i];
        double nr, ni;
        if (l == 0) {  // Phi_1 = -i y
          nr = yi;
          ni = -yr;
          accr = fma(cf.a[1], nr, cf.a[0] * cur.x);
          acci = fma(cf.a[1], ni, cf.a[0] * cur.y);
        } else {       // Phi_{l+1} = -2i y + Phi_{l-1}
          nr = fma(2.0, yi, pvr);
          ni = fma(-2.0, yr, pvi);
          accr = fma(cf.a[l + 1], nr, accr);
          acci = fma(cf.a[l + 1], ni, acci);
        }
        pvr = cur.x;
        pvi = cur.y;
        bad |= !(nr * nr + ni * ni <= bound2);  // |T_l(Omega~) x| <= |x| inside the bounds
        if (l == L - 1) {  // X_m = e^{-i beta h} acc
          nr = ph_re * accr - ph_im * acci;
          ni = ph_re * acci + ph_im * accr;
        }
        if (C > 1) {
          for (int c = 0; c < C; ++c) st_cluster_f64x2(&phi[buf ^ 1][i], (unsigned)c, nr, ni);
        } else {
          phi[buf ^ 1][i] = make_double2(nr, ni);
        }
      }
      if (C > 1) cluster_sync_all();
      else __syncthreads();
      buf ^= 1;
    }
  }
  if (own) {
    xr[(size_t)j * n + i] = phi[buf][i].x;
    xi[(size_t)j * n + i] = phi[buf][i].y;
  }
  if (bad) atomicOr(status, FQ_BIT_BOUND);
  if (C > 1) cluster_sync_all();  // no CTA leaves while a peer could still address its memory
}

__device__ __forceinline__ void st_cluster_f32x4(const void* local, unsigned rank, float4 v) {
  const unsigned la = (unsigned)__cvta_generic_to_shared(local);
  unsigned ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(la), "r"(rank));
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(ra), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
               : "memory");
}

__device__ __forceinline__ dflc dflc_shfl_xor(dflc a, int o) {
  return {make_float2(__shfl_xor_sync(0xffffffffu, a.h.x, o), __shfl_xor_sync(0xffffffffu, a.h.y, o)),
          make_float2(__shfl_xor_sync(0xffffffffu, a.l.x, o), __shfl_xor_sync(0xffffffffu, a.l.y, o))};
}

// The chain of k_dense_resident in double-float arithmetic: S, A as FP32 pairs [nsteps][n][n]
// (float2 = (hi, lo)), the state as packed complex pairs in shared memory.
template <int ROWS, int KG>
__global__ void __launch_bounds__(ROWS* KG)
    k_dense_resident_dfl(const float2* __restrict__ S, const float2* __restrict__ A, int n, int nsteps, int L, int C,
                         DrCoef cf, double ph_re, double ph_im, double bound2, double* xr, double* xi,
                         unsigned* status) {
  constexpr int NT = ROWS * KG;
  constexpr int NV = KG * DR_KPT;
  __shared__ dflc phi[2][NV];
  const int t = threadIdx.x, rl = t / KG, g = t % KG;
  const unsigned rank = C > 1 ? cluster_rank() : 0u;
  const int j = blockIdx.x / C;
  const int i = (int)rank * ROWS + rl;
  const bool own = g == 0 && i < n;
  const dflc zc = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  for (int q = t; q < 2 * NV; q += NT) {
    const int b = q / NV, k = q % NV;
    dflc v = zc;
    if (b == 0 && k < n) {
      const dfl r = dfl_of(xr[(size_t)j * n + k]), m = dfl_of(xi[(size_t)j * n + k]);
      v = {make_float2(r.h, m.h), make_float2(r.l, m.l)};
    }
    phi[b][k] = v;
  }
  __syncthreads();
  if (C > 1) cluster_sync_all();
  const size_t nn = (size_t)n * n;
  const dfl ph_c = dfl_of(ph_re), ph_s = dfl_of(ph_im);
  int buf = 0;
  bool bad = false;
  for (int m = 0; m < nsteps; ++m) {
    dfl s[DR_KPT], a[DR_KPT];
#pragma unroll
    for (int q = 0; q < DR_KPT; ++q) {
      const int k = g + KG * q;
      const bool ok = i < n && k < n;
      const float2 sv = ok ? S[m * nn + (size_t)i * n + k] : make_float2(0.f, 0.f);
      const float2 av = ok ? A[m * nn + (size_t)i * n + k] : make_float2(0.f, 0.f);
      s[q] = dfl{sv.x, sv.y};
      a[q] = dfl{av.x, av.y};
    }
    dflc acc = zc, pv = zc;
    for (int l = 0; l < L; ++l) {
      dflc ys = zc, ya = zc;  // S phi and i A phi, two independent chains
#pragma unroll
      for (int q = 0; q < DR_KPT; ++q) {
        const dflc v = phi[buf][g + KG * q];
        ys = dflc_fma(s[q], v, ys);
        ya = dflc_ifma2(a[q], v, ya);
      }
      dflc y = dflc_add(ys, ya);
#pragma unroll
      for (int o = KG / 2; o > 0; o >>= 1) y = dflc_add(y, dflc_shfl_xor(y, o));
      if (own) {
        const dflc cur = phi[buf][i];
        // -i y (first product) or -2i y + phi_{l-1}: (y_im, -y_re) scaled exactly
        const float sc = l == 0 ? 1.f : 2.f;
        const dflc my = {make_float2(sc * y.h.y, -sc * y.h.x), make_float2(sc * y.l.y, -sc * y.l.x)};
        const dflc nx = l == 0 ? my : dflc_add(my, pv);
        const dfl al = dfl_of(cf.a[l + 1]);
        acc = l == 0 ? dflc_fma(al, nx, dflc_fma(dfl_of(cf.a[0]), cur, zc)) : dflc_fma(al, nx, acc);
        pv = cur;
        const double nr = (double)nx.h.x + (double)nx.l.x, ni = (double)nx.h.y + (double)nx.l.y;
        bad |= !(nr * nr + ni * ni <= bound2);
        dflc out = nx;
        if (l == L - 1) out = dflc_ifma2(ph_s, acc, dflc_fma(ph_c, acc, zc));  // (ph_re + i ph_im) acc
        const float4 w = make_float4(out.h.x, out.h.y, out.l.x, out.l.y);
        if (C > 1) {
          for (int c = 0; c < C; ++c) st_cluster_f32x4(&phi[buf ^ 1][i], (unsigned)c, w);
        } else {
          phi[buf ^ 1][i] = out;
        }
      }
      if (C > 1) cluster_sync_all();
      else __syncthreads();
      buf ^= 1;
    }
  }
  if (own) {
    const dflc v = phi[buf][i];
    xr[(size_t)j * n + i] = (double)v.h.x + (double)v.l.x;
    xi[(size_t)j * n + i] = (double)v.h.y + (double)v.l.y;
  }
  if (bad) atomicOr(status, FQ_BIT_BOUND);
  if (C > 1) cluster_sync_all();
}

// S, A of a chunk as FP32 pairs
__global__ void k_to_dfl(const double* __restrict__ S, const double* __restrict__ A, size_t count, float2* Sd,
                         float2* Ad) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < count; q += (size_t)gridDim.x * blockDim.x) {
    const dfl s = dfl_of(S[q]), a = dfl_of(A[q]);
    Sd[q] = make_float2(s.h, s.l);
    Ad[q] = make_float2(a.h, a.l);
  }
}

// Omega~ of steps m0 .. m0+nsteps-1 (order 4, Eq. 11 on Omega_m/h): S = sa H0 + sb H1 - sbeta 1,
// A = sc [H0,H1], scalars from the plan's device copy (sa | sb | sc, M each).
__global__ void k_omega_dense_steps(const double* __restrict__ h0, const double* __restrict__ h1,
                                    const double* __restrict__ k, int n, const double* __restrict__ scal, int M,
                                    int m0, int nsteps, double sbeta, double* S, double* A) {
  const size_t nn = (size_t)n * n, total = nn * nsteps;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)(q / nn);
    const size_t e = q % nn;
    const int i = (int)(e / n), jj = (int)(e % n);
    const double sa = scal[m0 + m], sb = scal[M + m0 + m], sc = scal[2 * M + m0 + m];
    S[q] = sa * h0[e] + sb * h1[e] - (i == jj ? sbeta : 0.0);
    A[q] = sc * k[e];
  }
}

template <int ROWS, int KG>
cudaError_t launch_resident(const fq_plan* p, const double* S, const double* A, const float2* Sd, const float2* Ad,
                            int nsteps, double* xr, double* xi, int nc, cudaStream_t s) {
  const int C = (p->n + ROWS - 1) / ROWS;
  DrCoef cf{};
  for (int l = 0; l <= p->L; ++l) cf.a[l] = p->cheb[l];
  const double bound2 = 1.0 + 1e-9;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(nc * C));
  cfg.blockDim = dim3(ROWS * KG);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  if (C > 1) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  if (p->precision == FQ_DF32)
    return cudaLaunchKernelEx(&cfg, k_dense_resident_dfl<ROWS, KG>, (const float2*)Sd, (const float2*)Ad, p->n, nsteps,
                              p->L, C, cf, p->phase_re, p->phase_im, bound2, xr, xi, p->d_status);
  return cudaLaunchKernelEx(&cfg, k_dense_resident<ROWS, KG>, S, A, p->n, nsteps, p->L, C, cf, p->phase_re,
                            p->phase_im, bound2, xr, xi, p->d_status);
}

}  // namespace

bool fq_dense_resident_supported(int n, int L) { return n >= 1 && n <= DR_MAXN && L >= 1 && L <= DR_MAXL; }

size_t fq_dense_resident_omega_count(int n, int nsteps) {
  // FP64 S (or A) of a chunk, and room for its FP32-pair copy (FQ_DF32) after it
  return 2 * (size_t)std::min(nsteps, DR_CHUNK) * n * n;
}

fq_status fq_dense_resident_chain(const fq_plan* p, double* xr, double* xi, int nc, int m_begin, int m_end,
                                  double* S, double* A, cudaStream_t s) {
  const int n = p->n;
  const size_t nn = (size_t)n * n;
  for (int m0 = m_begin; m0 < m_end; m0 += DR_CHUNK) {
    const int cnt = std::min(DR_CHUNK, m_end - m0);
    if (p->order == 6) {
      const double inv = 1.0 / (p->h * p->delta_e);
      for (int m = 0; m < cnt; ++m) {
        double c[FQ_M6_TERMS];
        for (int q = 0; q < FQ_M6_TERMS; ++q) c[q] = p->coef6[(size_t)(m0 + m) * FQ_M6_TERMS + q] * inv;
        fq_launch_omega6_f64(p, c, S + m * nn, A + m * nn, s);
      }
    } else {
      const size_t total = nn * cnt;
      const int grid = (int)std::min<size_t>((total + 255) / 256, 152 * 16);
      k_omega_dense_steps<<<grid, 256, 0, s>>>(p->d_h0, p->d_h1, p->d_k, n, p->d_scal, p->steps, m0, cnt, p->sbeta,
                                               S, A);
    }
    // FQ_DF32: FP32-pair copies in the second half of each region
    const size_t cap = (size_t)std::min(m_end - m_begin, DR_CHUNK);  // chunk size the regions were sized for
    float2* Sd = reinterpret_cast<float2*>(S + cap * nn);
    float2* Ad = reinterpret_cast<float2*>(A + cap * nn);
    if (p->precision == FQ_DF32) {
      const size_t total = nn * cnt;
      k_to_dfl<<<(int)std::min<size_t>((total + 255) / 256, 152 * 16), 256, 0, s>>>(S, A, total, Sd, Ad);
    }
    // double-float: CTAs of 16 rows, a cluster of up to eight per state (the products are cheap
    // on the FP32 pipes; more SMs share each product)
    cudaError_t e;
    if (p->precision == FQ_DF32 && n <= 64) e = launch_resident<16, 8>(p, S, A, Sd, Ad, cnt, xr, xi, nc, s);
    else if (p->precision == FQ_DF32) e = launch_resident<16, 16>(p, S, A, Sd, Ad, cnt, xr, xi, nc, s);
    else if (n <= 64) e = launch_resident<DR_ROWS, 8>(p, S, A, Sd, Ad, cnt, xr, xi, nc, s);
    else e = launch_resident<DR_ROWS, 16>(p, S, A, Sd, Ad, cnt, xr, xi, nc, s);
    if (e != cudaSuccess) return fq_cuda_fail(e, "dense resident chain");
  }
  return FQ_OK;
}
