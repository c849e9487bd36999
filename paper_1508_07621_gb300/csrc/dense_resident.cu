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
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

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
template <int KG>
__global__ void __launch_bounds__(DR_ROWS* KG)
    k_dense_resident(const double* __restrict__ S, const double* __restrict__ A, int n, int nsteps, int L, int C,
                     DrCoef cf, double ph_re, double ph_im, double bound2, double* xr, double* xi,
                     unsigned* status) {
  constexpr int NT = DR_ROWS * KG;
  constexpr int NV = KG * DR_KPT;  // vector length held per buffer (>= n)
  __shared__ double2 phi[2][NV];
  const int t = threadIdx.x, rl = t / KG, g = t % KG;
  const unsigned rank = C > 1 ? cluster_rank() : 0u;
  const int j = blockIdx.x / C;  // the state this cluster carries
  const int i = (int)rank * DR_ROWS + rl;
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

template <int KG>
cudaError_t launch_resident(const fq_plan* p, const double* S, const double* A, int nsteps, int C, double* xr,
                            double* xi, int nc, cudaStream_t s) {
  DrCoef cf{};
  for (int l = 0; l <= p->L; ++l) cf.a[l] = p->cheb[l];
  const double bound2 = 1.0 + 1e-9;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(nc * C));
  cfg.blockDim = dim3(DR_ROWS * KG);
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
  return cudaLaunchKernelEx(&cfg, k_dense_resident<KG>, S, A, p->n, nsteps, p->L, C, cf, p->phase_re, p->phase_im,
                            bound2, xr, xi, p->d_status);
}

}  // namespace

bool fq_dense_resident_supported(int n, int L) { return n >= 1 && n <= DR_MAXN && L >= 1 && L <= DR_MAXL; }

size_t fq_dense_resident_omega_count(int n, int nsteps) {
  return (size_t)std::min(nsteps, DR_CHUNK) * n * n;
}

fq_status fq_dense_resident_chain(const fq_plan* p, double* xr, double* xi, int nc, int m_begin, int m_end,
                                  double* S, double* A, cudaStream_t s) {
  const int n = p->n;
  const int C = (n + DR_ROWS - 1) / DR_ROWS;
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
    cudaError_t e = n <= 64 ? launch_resident<8>(p, S, A, cnt, C, xr, xi, nc, s)
                            : launch_resident<16>(p, S, A, cnt, C, xr, xi, nc, s);
    if (e != cudaSuccess) return fq_cuda_fail(e, "dense resident chain");
  }
  return FQ_OK;
}
