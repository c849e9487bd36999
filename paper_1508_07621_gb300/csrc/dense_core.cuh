// FP64 SIMT tile of the dense Chebyshev product used by the forward term, the adjoint term and
// the gradient dot products:  Y^T[j][i] = sum_k X[j][k] (S[i][k] + i A[i][k])  for the
// BJ x BI tile (j0.., i0..) of an nc x n block of state rows X.  S is real symmetric, A real
// antisymmetric (HAS_A = false: A == 0, a real operator).  (BJ/TJ) x (BI/TI) threads, TJ x TI
// complex outputs per thread, K staged through shared memory in BK slices.
#pragma once

template <int BJ, int BI, int BK, int TJ, int TI, bool HAS_A>
__device__ __forceinline__ void dense_tile_f64(const double* __restrict__ S, const double* __restrict__ A, int n,
                                               const double* __restrict__ x_re, const double* __restrict__ x_im,
                                               int nc, int j0, int i0, double (&yr)[TJ][TI], double (&yi)[TJ][TI]) {
  constexpr int NTX = BI / TI, NTY = BJ / TJ, NT = NTX * NTY;
  __shared__ double sPr[BK][BJ + 1], sPi[BK][BJ + 1], sS[BK][BI + 1], sA[HAS_A ? BK : 1][BI + 1];
  const int tx = threadIdx.x % NTX, ty = threadIdx.x / NTX;
#pragma unroll
  for (int a = 0; a < TJ; ++a)
#pragma unroll
    for (int b = 0; b < TI; ++b) yr[a][b] = yi[a][b] = 0.0;
  for (int k0 = 0; k0 < n; k0 += BK) {
    for (int q = threadIdx.x; q < BJ * BK; q += NT) {
      int r = q / BK, kk = q % BK, j = j0 + r, k = k0 + kk;
      bool ok = j < nc && k < n;
      sPr[kk][r] = ok ? x_re[(size_t)j * n + k] : 0.0;
      sPi[kk][r] = ok ? x_im[(size_t)j * n + k] : 0.0;
    }
    for (int q = threadIdx.x; q < BI * BK; q += NT) {
      int r = q / BK, kk = q % BK, i = i0 + r, k = k0 + kk;
      bool ok = i < n && k < n;
      sS[kk][r] = ok ? S[(size_t)i * n + k] : 0.0;
      if (HAS_A) sA[kk][r] = ok ? A[(size_t)i * n + k] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      double pr[TJ], pi[TJ], s[TI], a[TI];
#pragma unroll
      for (int q = 0; q < TJ; ++q) { pr[q] = sPr[kk][ty * TJ + q]; pi[q] = sPi[kk][ty * TJ + q]; }
#pragma unroll
      for (int q = 0; q < TI; ++q) {
        s[q] = sS[kk][tx * TI + q];
        a[q] = HAS_A ? sA[HAS_A ? kk : 0][tx * TI + q] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < TJ; ++u)
#pragma unroll
        for (int v = 0; v < TI; ++v) {
          if (HAS_A) {
            yr[u][v] = fma(pr[u], s[v], fma(-pi[u], a[v], yr[u][v]));
            yi[u][v] = fma(pi[u], s[v], fma(pr[u], a[v], yi[u][v]));
          } else {
            yr[u][v] = fma(pr[u], s[v], yr[u][v]);
            yi[u][v] = fma(pi[u], s[v], yi[u][v]);
          }
        }
    }
    __syncthreads();
  }
}
