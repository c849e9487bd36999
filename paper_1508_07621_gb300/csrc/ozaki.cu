// Forward chain of the FP64 emulation (FQ_OZAKI, kernels in ozaki_core.cuh): per step the
// fixed-point slices of Omega~_m, then L terms of Eq. 10 through k_oz_term whose
// FP64 epilogue applies the recurrence, the Bessel accumulation of Eq. 12 and the step phase;
// each new state block is sliced again (its row scales need whole rows).
#include "ozaki_core.cuh"

namespace {

struct OzWs {
  __nv_bfloat16* left;   // OZ_S slices [ncp][2 np]
  __nv_bfloat16* right;  // OZ_S slices [3 np][np]
  int* es;               // [ncp]
  int* et;               // [np]
  double* m[3][2];       // FP64 state masters [nc][n], planar
  int np, ncp;
  size_t astride, rstride;
};

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

OzOmega omega_args(const fq_plan* p, int m) {
  OzOmega a{};
  a.sbeta = p->sbeta;
  if (p->order == 6) {
    static const int anti[FQ_M6_TERMS] = {0, 0, 1, 0, 0, 1, 1, 1, 1, 0, 0};
    const size_t nn = (size_t)p->n * p->n;
    const double inv = 1.0 / (p->h * p->delta_e);
    a.terms = FQ_M6_TERMS;
    a.m[0] = p->d_h0;
    a.m[1] = p->d_h1;
    a.m[2] = p->d_k;
    for (int q = 0; q < 8; ++q) a.m[3 + q] = p->d_cm + q * nn;
    for (int q = 0; q < FQ_M6_TERMS; ++q) {
      a.c[q] = p->coef6[(size_t)m * FQ_M6_TERMS + q] * inv;
      a.anti[q] = anti[q];
    }
  } else {
    a.terms = 3;
    a.m[0] = p->d_h0;
    a.m[1] = p->d_h1;
    a.m[2] = p->d_k;
    a.c[0] = p->sa[m];
    a.c[1] = p->sb[m];
    a.c[2] = p->sc[m];
    a.anti[2] = 1;
  }
  return a;
}

}  // namespace

size_t fq_ozaki_workspace(const fq_plan* p, int nc, void* base, void* out) {
  OzWs w{};
  w.np = (p->n + 127) & ~127;
  w.ncp = (nc + BM - 1) / BM * BM;
  w.astride = (size_t)w.ncp * 2 * w.np;
  w.rstride = (size_t)3 * w.np * w.np;
  char* b = (char*)base;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* q = b ? b + off : nullptr;
    off += up256(bytes);
    return q;
  };
  w.left = (__nv_bfloat16*)take(sizeof(__nv_bfloat16) * OZ_S * w.astride);
  w.right = (__nv_bfloat16*)take(sizeof(__nv_bfloat16) * OZ_S * w.rstride);
  w.es = (int*)take(sizeof(int) * w.ncp);
  w.et = (int*)take(sizeof(int) * w.np);
  for (int q = 0; q < 3; ++q)
    for (int r = 0; r < 2; ++r) w.m[q][r] = (double*)take(sizeof(double) * (size_t)nc * p->n);
  if (out) *(OzWs*)out = w;
  return off;
}

fq_status fq_ozaki_propagate(fq_plan* p, const double* x0, double* x, int nc, int m_begin, int m_end, int identity,
                             int transpose_out, void* ws, cudaStream_t s) {
  fq_status st = encode_fn();
  if (st != FQ_OK) return st;
  OzWs w;
  fq_ozaki_workspace(p, nc, ws, &w);
  const int n = p->n, L = p->L;
  OzMaps maps;
  for (int q = 0; q < OZ_S; ++q) {
    if ((st = make_map(&maps.a[q], w.left + q * w.astride, w.ncp, 2 * w.np, BM, OZ_BKE)) != FQ_OK) return st;
    if ((st = make_map(&maps.r[q], w.right + q * w.rstride, 3 * w.np, w.np, 3 * OZ_BN, OZ_BKE)) != FQ_OK) return st;
  }
  static std::atomic<unsigned> attr_set{0};
  if (fq_first_on_device(attr_set)) {
    cudaError_t e = cudaFuncSetAttribute(k_oz_term, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)OzCfg::SMEM);
    if (e != cudaSuccess) return fq_cuda_fail(e, "Ozaki kernel shared-memory attribute");
  }
  fq_blk<double> b0{w.m[0][0], w.m[0][1]};
  if (identity) fq_launch_identity_f64(b0, nc, n, n, s);
  else fq_launch_load_states(x0, b0, nc, n, n, s);
  int xb = 0;
  if (m_end > m_begin)
    k_oz_slice_left<<<w.ncp, 256, 0, s>>>(w.m[0][0], w.m[0][1], 1.0, 0.0, nullptr, nullptr, n, nc, w.np, w.astride,
                                          w.left, w.es);
  const int tiles_i = w.np / OZ_BN, tiles_j = w.ncp / BM;
  const int nk = w.np / OZ_BKE;
  fq_term t{};
  t.coef0 = p->cheb[0];
  t.ph_re = p->phase_re;
  t.ph_im = p->phase_im;
  t.bound2 = 1.0 + 1e-9;
  t.status = p->d_status;
  for (int m = m_begin; m < m_end; ++m) {
    k_oz_omega<<<w.np, 256, 0, s>>>(omega_args(p, m), n, w.np, w.rstride, w.right, w.et);
    int cur = xb, nxt = (xb + 1) % 3, acc = (xb + 2) % 3, prv = -1;
    for (int l = 0; l < L; ++l) {
      t.first = l == 0;
      t.last = l == L - 1;
      t.coef = p->cheb[l + 1];
      const int out = l == 0 ? nxt : prv;
      OzEpi e{};
      e.n = n;
      e.nc = nc;
      e.cur_re = w.m[cur][0];
      e.cur_im = w.m[cur][1];
      e.prev_re = prv >= 0 ? w.m[prv][0] : w.m[cur][0];
      e.prev_im = prv >= 0 ? w.m[prv][1] : w.m[cur][1];
      e.acc_re = w.m[acc][0];
      e.acc_im = w.m[acc][1];
      e.out_re = w.m[out][0];
      e.out_im = w.m[out][1];
      e.es = w.es;
      e.et = w.et;
      e.t = t;
      k_oz_term<<<tiles_i * tiles_j, OZ_THREADS, OzCfg::SMEM, s>>>(maps, nk, tiles_j, tiles_i,
                                                                                        w.np, e);
      if (!(t.last && m == m_end - 1))
        k_oz_slice_left<<<w.ncp, 256, 0, s>>>(w.m[out][0], w.m[out][1], 1.0, 0.0, nullptr, nullptr, n, nc, w.np,
                                              w.astride, w.left, w.es);
      if (t.last) {
        xb = out;
      } else {
        prv = cur;
        cur = out;
      }
    }
  }
  fq_blk<double> bx{w.m[xb][0], w.m[xb][1]};
  if (transpose_out) fq_launch_store_transpose_f64(bx, x, n, n, s);
  else fq_launch_store_states_f64(bx, x, nc, n, n, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fq_cuda_fail(e, "Ozaki kernels");
  return FQ_OK;
}
