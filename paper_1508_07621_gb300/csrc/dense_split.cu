// Split-precision dense Chebyshev chain (stages a2, a3, a5, a6, a8 on the tensor cores): per step
// the S and A slices of Omega~_m (FP64 arithmetic, Eqs. 11 and 14), then L terms of Eq. 10 through
// k_split_term (split_core.cuh) whose epilogue applies the recurrence, the Bessel accumulation
// of Eq. 12 and the step phase, and writes the next term's BF16 slices.
#include <vector>

#include "split_core.cuh"

namespace {

// Right operands of step m: S and A of Omega~_m = S + i A as NS BF16 slices [Np][Np] each (stage
// a2): S = sa H0 + sb H1 - sbeta 1, A = sc [H0,H1], formed in FP32 (omega_entry); zero outside
// N x N.
template <int NS>
__global__ void k_split_omega(const double* __restrict__ h0, const double* __restrict__ h1,
                              const double* __restrict__ k, int n, int np, float sa, float sb, float sc,
                              float sbeta, __nv_bfloat16* os, __nv_bfloat16* oa, size_t slice_stride) {
  const size_t total = (size_t)np * np;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(q / np), c = (int)(q % np);
    float S = 0.f, A = 0.f;
    if (i < n && c < n) {
      const size_t o = (size_t)i * n + c;
      omega_entry(h0[o], h1[o], k[o], i == c, sa, sb, sc, sbeta, S, A);
    }
    __nv_bfloat16 s1[NS], s2[NS];
    split_f32<NS>(S, s1);
    split_f32<NS>(A, s2);
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      os[t * slice_stride + q] = s1[t];
      oa[t * slice_stride + q] = s2[t];
    }
  }
}

// 6th order: S and A slices of Omega~ = sum_q c_q M_q (c already divided by h Delta E).
struct Omega6Split {
  const double* m[FQ_M6_TERMS];
  double c[FQ_M6_TERMS];
  double sbeta;
  int n, np;
};

template <int NS>
__global__ void k_split_omega6(Omega6Split a, __nv_bfloat16* os, __nv_bfloat16* oa, size_t slice_stride) {
  const size_t total = (size_t)a.np * a.np;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(q / a.np), c = (int)(q % a.np);
    double S = 0.0, A = 0.0;
    if (i < a.n && c < a.n) {
      const size_t o = (size_t)i * a.n + c;
      S = (i == c) ? -a.sbeta : 0.0;
      const int sym[6] = {0, 1, 3, 4, 9, 10}, anti[5] = {2, 5, 6, 7, 8};
#pragma unroll
      for (int t = 0; t < 6; ++t) S = fma(a.c[sym[t]], a.m[sym[t]][o], S);
#pragma unroll
      for (int t = 0; t < 5; ++t) A = fma(a.c[anti[t]], a.m[anti[t]][o], A);
    }
    __nv_bfloat16 s1[NS], s2[NS];
    split_f64<NS>(S, s1);
    split_f64<NS>(A, s2);
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      os[t * slice_stride + q] = s1[t];
      oa[t * slice_stride + q] = s2[t];
    }
  }
}


}  // namespace

// ------------------------------------------------------------------------- orchestration
static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t fq_split_workspace(const fq_plan* p, int nc, void* base, void* out) {
  const int NS = p->precision == FQ_BF16X6 ? 3 : 2;
  SplitWs w{};
  w.np = (p->n + 127) & ~127;  // whole output tiles for both tile widths
  w.kp = 2 * w.np;
  w.ldm = (p->n + 3) & ~3;
  w.bstride = (size_t)w.np * w.np;
  w.ncp = (nc + BM - 1) / BM * BM;  // left-operand rows padded to whole 128-row boxes (zeros)
  w.astride = (size_t)w.ncp * w.kp;
  char* b = (char*)base;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* q = b ? b + off : nullptr;
    off += up256(bytes);
    return q;
  };
  w.os = (__nv_bfloat16*)take(2 * NS * w.bstride);
  w.oa = (__nv_bfloat16*)take(2 * NS * w.bstride);
  w.a[0] = (__nv_bfloat16*)take(2 * NS * w.astride);
  w.a[1] = (__nv_bfloat16*)take(2 * NS * w.astride);
  for (int q = 0; q < 3; ++q)
    for (int r = 0; r < 2; ++r) w.m[q][r] = (float*)take(sizeof(float) * (size_t)nc * w.ldm);
  w.flags = (unsigned int*)take(sizeof(unsigned int) * CHAIN_MAXP * (size_t)(w.ncp / BM));
  if (out) *(SplitWs*)out = w;
  return off;
}

template <int NS, int BN, int BKE>
static fq_status run_split(fq_plan* p, const double* x0, double* x, int nc, int m_begin, int m_end, int identity,
                           int transpose_out, void* ws, cudaStream_t s) {
  using Cfg = SplitCfg<NS, BN, BKE, true>;
  fq_status st = encode_fn();
  if (st != FQ_OK) return st;
  SplitWs w;
  fq_split_workspace(p, nc, ws, &w);
  const int n = p->n, L = p->L;
  SplitMaps maps[2];  // left operand in a[0] or a[1]
  for (int v = 0; v < 2; ++v)
    for (int q = 0; q < NS; ++q) {
      if ((st = make_map(&maps[v].a[q], w.a[v] + q * w.astride, w.ncp, w.kp, BM, BKE)) != FQ_OK) return st;
      if ((st = make_map(&maps[v].os[q], w.os + q * w.bstride, w.np, w.np, BN, BKE)) != FQ_OK) return st;
      if ((st = make_map(&maps[v].oa[q], w.oa + q * w.bstride, w.np, w.np, BN, BKE)) != FQ_OK) return st;
    }
  static std::atomic<unsigned> attr_set{0};
  if (fq_first_on_device(attr_set)) {
    cudaError_t e = cudaFuncSetAttribute(k_split_persist<NS, BN, BKE, EPI_FWD, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
    if (e != cudaSuccess) return fq_cuda_fail(e, "split kernel shared-memory attribute");
  }
  const int sms = fq_sm_count();
  // left-operand slices are only ever written for rows < nc and columns < n: zero the padding
  cudaMemsetAsync(w.a[0], 0, sizeof(__nv_bfloat16) * NS * w.astride, s);
  cudaMemsetAsync(w.a[1], 0, sizeof(__nv_bfloat16) * NS * w.astride, s);
  k_split_init<NS><<<grid_1d((size_t)nc * w.kp), 256, 0, s>>>(identity ? nullptr : (const double2*)x0, n, nc, w.ldm,
                                                               w.np, w.kp, w.m[0][0], w.m[0][1], w.a[0], w.astride);
  const int tiles_i = w.np / BN, tiles_j = (nc + BM - 1) / BM;
  // persistent: at most one CTA per SM, or the batch's share of them (lanes' products run side by side)
  const dim3 grid(std::min(tiles_i * tiles_j, p->grid_cap > 0 ? std::min(p->grid_cap, sms) : sms));
  // K runs to N rounded up to the stage depth: the operands' columns beyond N are zero
  const int nk = (n + BKE - 1) / BKE;
  int xb = 0, av = 0;  // FP32 master holding psi_0 / X, left-operand buffer holding its slices
  fq_term t{};
  t.coef0 = p->cheb[0];
  t.ph_re = p->phase_re;
  t.ph_im = p->phase_im;
  t.bound2 = 1.0 + 2e-3;
  t.status = p->d_status;
  for (int m = m_begin; m < m_end; ++m) {
    if (p->order == 6) {
      Omega6Split a;
      const size_t nn = (size_t)n * n;
      a.m[0] = p->d_h0;
      a.m[1] = p->d_h1;
      a.m[2] = p->d_k;
      for (int q = 0; q < 8; ++q) a.m[3 + q] = p->d_cm + q * nn;
      const double inv = 1.0 / (p->h * p->delta_e);
      for (int q = 0; q < FQ_M6_TERMS; ++q) a.c[q] = p->coef6[(size_t)m * FQ_M6_TERMS + q] * inv;
      a.sbeta = p->sbeta;
      a.n = n;
      a.np = w.np;
      k_split_omega6<NS><<<grid_1d(w.bstride), 256, 0, s>>>(a, w.os, w.oa, w.bstride);
    } else {
      k_split_omega<NS><<<grid_1d(w.bstride), 256, 0, s>>>(p->d_h0, p->d_h1, p->d_k, n, w.np, (float)p->sa[m],
                                                           (float)p->sb[m], (float)p->sc[m], (float)p->sbeta,
                                                           w.os, w.oa, w.bstride);
    }
    // the step's L terms: their epilogues and left-operand buffers, then one cooperative chain
    // launch (a term's tiles start as soon as the previous term has finished their row block), or
    // one persistent launch per term where a chain cannot run (a capturing stream, L > CHAIN_MAXP)
    std::vector<SplitEpi> eps(L);
    std::vector<int> left_of(L);
    int cur = xb, nxt = (xb + 1) % 3, acc = (xb + 2) % 3, prv = -1;
    for (int l = 0; l < L; ++l) {
      t.first = l == 0;
      t.last = l == L - 1;
      t.coef = p->cheb[l + 1];
      const int out = l == 0 ? nxt : prv;
      SplitEpi& e = eps[l];
      e = SplitEpi{};
      e.n = n;
      e.nc = nc;
      e.ldm = w.ldm;
      e.np = w.np;
      e.kp = w.kp;
      e.cur_re = w.m[cur][0];
      e.cur_im = w.m[cur][1];
      e.prev_re = prv >= 0 ? w.m[prv][0] : w.m[cur][0];
      e.prev_im = prv >= 0 ? w.m[prv][1] : w.m[cur][1];
      e.acc_re = w.m[acc][0];
      e.acc_im = w.m[acc][1];
      e.out_re = w.m[out][0];
      e.out_im = w.m[out][1];
      e.slice_out = w.a[av ^ 1];
      e.slice_stride = w.astride;
      e.t = t;
      left_of[l] = av;
      av ^= 1;
      if (t.last) {
        xb = out;
      } else {
        prv = cur;
        cur = out;
      }
    }
    st = FQ_EUNSUPPORTED;
    if (L <= CHAIN_MAXP) {
      ChainArgs ch{};
      ch.rmaps = maps[0];
      ch.nprod = L;
      ch.nk = nk;
      ch.tiles_j = tiles_j;
      ch.tiles_i = tiles_i;
      ch.flags = w.flags;
      for (int l = 0; l < L; ++l) {
        ch.epi[l] = eps[l];
        for (int q = 0; q < NS; ++q) ch.left[l][q] = maps[left_of[l]].a[q];
      }
      cudaError_t ce = cudaMemsetAsync(w.flags, 0, sizeof(unsigned int) * (size_t)L * tiles_j, s);
      if (ce != cudaSuccess) return fq_cuda_fail(ce, "chain counters");
      st = launch_chain<NS, BN, BKE, EPI_FWD, true>(ch, s);
      if (st != FQ_OK && st != FQ_EUNSUPPORTED) return st;
    }
    if (st == FQ_EUNSUPPORTED)
      for (int l = 0; l < L; ++l)
        k_split_persist<NS, BN, BKE, EPI_FWD, true><<<grid, PTHREADS, Cfg::SMEM, s>>>(maps[left_of[l]], nk, tiles_j,
                                                                                     tiles_i, eps[l]);
  }
  fq_blk<float> bx{w.m[xb][0], w.m[xb][1]};
  if (x == nullptr) {
    // autotuning runs time the chain only
  } else if (transpose_out) {
    fq_launch_store_transpose_f32(bx, x, n, w.ldm, s);
  } else {
    fq_launch_store_states_f32(bx, x, nc, n, w.ldm, s);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fq_cuda_fail(e, "split-precision kernels");
  return FQ_OK;
}

fq_status fq_split_propagate(fq_plan* p, const double* x0, double* x, int nc, int m_begin, int m_end, int identity,
                             int transpose_out, void* ws, cudaStream_t s) {
  // (slices, tile width, K per stage): 64-byte swizzle stages where 128-byte ones would not fit
  // more than two stages in shared memory
  const bool wide = p->tile_n == 128;
  if (p->precision == FQ_BF16X6)
    return wide ? run_split<3, 128, 32>(p, x0, x, nc, m_begin, m_end, identity, transpose_out, ws, s)
                : run_split<3, 64, 32>(p, x0, x, nc, m_begin, m_end, identity, transpose_out, ws, s);
  if (wide) return run_split<2, 128, 32>(p, x0, x, nc, m_begin, m_end, identity, transpose_out, ws, s);
  return p->tile_k == 32 ? run_split<2, 64, 32>(p, x0, x, nc, m_begin, m_end, identity, transpose_out, ws, s)
                         : run_split<2, 64, 64>(p, x0, x, nc, m_begin, m_end, identity, transpose_out, ws, s);
}

// Times each tile shape on two steps of the identity block and keeps the fastest: output widths
// 64 and 128, and for 64-wide BF16X3 tiles K stages of 64 or 32 elements (two stages of 96 KB or
// four of 48 KB); each shape runs as many stages as fit in shared memory.
static fq_status floquet_autotune_body(fq_plan* p, void* ws, size_t bytes, void* stream, int32_t* tile_n) {
  if (!p) {
    fq_set_error("floquet_autotune: NULL plan");
    return FQ_EINVAL;
  }
  if (p->path != PATH_DENSE_SPLIT) {
    if (tile_n) *tile_n = 0;
    return FQ_OK;
  }
  if (!ws || bytes < floquet_workspace_size(p, p->n) || ((uintptr_t)ws & 255)) {
    fq_set_error("floquet_autotune: workspace must be floquet_workspace_size(plan, N) bytes, 256-byte aligned");
    return FQ_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int steps = p->steps < 2 ? p->steps : 2;
  struct Shape {
    int n, k;
  };
  std::vector<Shape> cand = {{64, 0}, {128, 0}};
  if (p->precision != FQ_BF16X6) cand.push_back({64, 32});
  float best = 1e30f;
  Shape pick = cand[0];
  const Shape before{p->tile_n, p->tile_k};
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  fq_status st = e == cudaSuccess ? FQ_OK : fq_cuda_fail(e, "autotune events");
  for (const Shape& c : cand) {
    if (st != FQ_OK) break;
    p->tile_n = c.n;
    p->tile_k = c.k;
    st = fq_split_propagate(p, nullptr, nullptr, p->n, 0, steps, 1, 0, ws, s);  // warm-up
    if (st != FQ_OK) break;
    cudaEventRecord(a, s);
    st = fq_split_propagate(p, nullptr, nullptr, p->n, 0, steps, 1, 0, ws, s);
    if (st != FQ_OK) break;
    cudaEventRecord(b, s);
    if ((e = cudaEventSynchronize(b)) != cudaSuccess) {
      st = fq_cuda_fail(e, "autotune");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (ms < best) {
      best = ms;
      pick = c;
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  p->tile_n = st == FQ_OK ? pick.n : before.n;  // on failure the plan keeps the shape it had
  p->tile_k = st == FQ_OK ? pick.k : before.k;
  if (st == FQ_OK && tile_n) *tile_n = pick.n;
  return st;
}

extern "C" fq_status floquet_autotune(fq_plan* p, void* ws, size_t bytes, void* stream, int32_t* tile_n) {
  return fq_guard("floquet_autotune", [&] { return floquet_autotune_body(p, ws, bytes, stream, tile_n); });
}
