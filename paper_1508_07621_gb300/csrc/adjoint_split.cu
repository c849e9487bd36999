// floquet_grad for BF16X3 / BF16X6 plans: the reverse-mode chain of adjoint.cu (loss
// L = 1 - |Tr(W^+ U_T)|^2 / N^2, Clenshaw-form adjoint of Eqs. 10 and 12, dL/df_m from the kept
// forward Chebyshev vectors) with every N x N x N product on the tensor cores (k_split_term).
//
// Piecewise-constant f makes Omega~_m = (H0 + f_m H1 - beta) / Delta E real symmetric, so each
// product is Y = X . S^T on the planar (re, im) state rows with a real right operand: two MMA
// streams instead of four.  States stay FP32 masters between products, and every product reads
// the NS BF16 slices its producer's epilogue wrote:
//   forward term   (EPI_FWD): psi_{l+1} = -2i Y + psi_{l-1}, acc += a_{l+1} psi_{l+1}, phase;
//   adjoint term   (EPI_ADJ): bbar_l = conj(e^{-i beta h}) a_l G + i cw Omega~ bbar_{l+1} + bbar_{l+2}
//                             (cw = 2, and 1 for l = 0);
//   gradient dot   (EPI_DOT): D_l = <bbar_l, E psi_{l-1}> with E = H1 / Delta E, per-CTA partials;
//   dL/df_m = 2 Re sum_l w_l D_l  (w_1 = -i, w_l = -2i).
// Memory: FP32 masters of X every s = checkpoint_stride steps; each segment is recomputed once
// with the slices of every psi_l kept (they are the left operands of the dot products) and then
// walked backward.  The slots are stored slice-major ([slice][slot][row][k]) and bbar_1..bbar_L
// of a step are kept as one stacked block, so the L gradient dots of a step run as one GEMM over
// L x Np stacked rows.
#include <vector>

#include "split_core.cuh"

namespace {

int grid_n(size_t total) { return (int)std::min<size_t>(std::max<size_t>((total + 255) / 256, 1), 152 * 32); }

// NS slices [np][np] of the real matrix ((h0 ? h0 : 0) + c1 h1) * inv - shift 1, c1 = f[m] (or 1
// without f); zero outside N x N.  FP64 arithmetic.
template <int NS>
__global__ void k_real_slices(const double* __restrict__ h0, const double* __restrict__ h1,
                              const double* __restrict__ f, int m, double inv, double shift, int n, int np,
                              __nv_bfloat16* out, size_t stride) {
  const double c1 = f ? f[m] : 1.0;
  const size_t total = (size_t)np * np;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(q / np), c = (int)(q % np);
    double v = 0.0;
    if (i < n && c < n) {
      const size_t o = (size_t)i * n + c;
      v = ((h0 ? h0[o] : 0.0) + c1 * h1[o]) * inv - (i == c ? shift : 0.0);
    }
    __nv_bfloat16 sl[NS];
    split_f64<NS>(v, sl);
#pragma unroll
    for (int t = 0; t < NS; ++t) out[t * stride + q] = sl[t];
  }
}

// out = c * in (in NULL: the identity rows) on nc x n FP32 planar masters (row stride ldm): FP32
// copy (out_re NULL: none) and NS slices [.][kp] (re at column c, im at column np + c).
template <int NS>
__global__ void k_scale_slices(const float* __restrict__ in_re, const float* __restrict__ in_im, float cr, float ci,
                               float* out_re, float* out_im, int nc, int n, int ldm, int np, int kp,
                               __nv_bfloat16* sl, size_t stride) {
  const size_t total = (size_t)nc * n;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(q / n), c = (int)(q % n);
    const size_t idx = (size_t)j * ldm + c;
    float a, b;
    if (in_re) {
      a = in_re[idx];
      b = in_im[idx];
    } else {
      a = j == c ? 1.f : 0.f;
      b = 0.f;
    }
    const float r = cr * a - ci * b, i = cr * b + ci * a;
    if (out_re) {
      out_re[idx] = r;
      out_im[idx] = i;
    }
    __nv_bfloat16 sr[NS], si[NS];
    split_f32<NS>(r, sr);
    split_f32<NS>(i, si);
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      sl[t * stride + (size_t)j * kp + c] = sr[t];
      sl[t * stride + (size_t)j * kp + np + c] = si[t];
    }
  }
}

// partial[j] = sum_i conj(W[i][j]) X^T[j][i]  (X^T rows = states, FP32 planar, stride ldm)
__global__ void k_trace_f32(const double2* __restrict__ W, const float* __restrict__ xr, const float* __restrict__ xi,
                            int n, int ldm, double2* partial) {
  const int j = blockIdx.x;
  double sr = 0.0, si = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double2 w = W[(size_t)i * n + j];
    const double a = xr[(size_t)j * ldm + i], b = xi[(size_t)j * ldm + i];
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

// G_M = -tau W / N^2 as rows: G^T[j][i] = G[i][j], FP32 planar masters
__global__ void k_seed_f32(const double2* __restrict__ W, const double2* __restrict__ tau, int n, int ldm, float* gr,
                           float* gi) {
  const double2 t = *tau;
  const double s = -1.0 / ((double)n * n);
  const size_t total = (size_t)n * n;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(q / n), i = (int)(q % n);
    const double2 w = W[(size_t)i * n + j];
    gr[(size_t)j * ldm + i] = (float)(s * (t.x * w.x - t.y * w.y));
    gi[(size_t)j * ldm + i] = (float)(s * (t.x * w.y + t.y * w.x));
  }
}

struct Master {
  float* re;
  float* im;
};

// Workspace of the split gradient (all offsets 256-byte aligned).
struct SplitGradWs {
  int ns, np, kp, ldm, ncp, nseg, nslots, ncta;
  size_t bstride, astride;
  __nv_bfloat16* S;       // Omega~_m slices
  __nv_bfloat16* E;       // E = H1 / Delta E slices
  __nv_bfloat16* lsl[2];  // left-operand ping-pong (forward sweep, adjoint terms)
  __nv_bfloat16* slots;   // psi_l slices of one recomputed segment: NS x nslots x [ncp][kp]
  Master f[5];            // FP32 masters: forward cur / prev / acc; adjoint G and the next G
  Master bbar;            // bbar_1 .. bbar_L of one step: L blocks of ncp rows (padding rows zero)
  float* ck_base;         // nseg checkpoints of X, each 2 planes [n][ldm]
  double2* partial;       // (L + 1) x ncta
  unsigned int* flags;    // chain counters [CHAIN_MAXP][row blocks]
  double2* tau_partial;   // n
  double2* tau;
  size_t slot_slice() const { return (size_t)nslots * astride; }  // elements between slot slices
  __nv_bfloat16* slot(int q) const { return slots + (size_t)q * astride; }
  Master bbar_block(int l) const {  // bbar_l, l = 1..L
    const size_t o = (size_t)(l - 1) * ncp * ldm;
    return Master{bbar.re + o, bbar.im + o};
  }
  Master ckpt(int k, int n) const {
    float* b = ck_base + (size_t)k * 2 * n * ldm;
    return Master{b, b + (size_t)n * ldm};
  }
};

size_t up(size_t x) { return (x + 255) & ~(size_t)255; }

size_t split_grad_layout(const fq_plan* p, void* base, SplitGradWs* out) {
  SplitGradWs w{};
  const int n = p->n, L = p->L, s = p->stride;
  w.ns = p->precision == FQ_BF16X6 ? 3 : 2;
  w.np = (n + 127) & ~127;
  w.kp = 2 * w.np;
  w.ldm = (n + 3) & ~3;
  w.ncp = w.np;
  w.nseg = (p->steps + s - 1) / s;
  w.nslots = s * L + 1;
  w.bstride = (size_t)w.np * w.np;
  w.astride = (size_t)w.ncp * w.kp;
  const int bn = p->tile_n == 128 ? 128 : 64;
  w.ncta = (w.np / bn) * (w.ncp / BM);
  char* b = (char*)base;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* q = b ? b + off : nullptr;
    off += up(bytes);
    return q;
  };
  const size_t plane = (size_t)n * w.ldm;
  w.S = (__nv_bfloat16*)take(2 * w.ns * w.bstride);
  w.E = (__nv_bfloat16*)take(2 * w.ns * w.bstride);
  w.lsl[0] = (__nv_bfloat16*)take(2 * w.ns * w.astride);
  w.lsl[1] = (__nv_bfloat16*)take(2 * w.ns * w.astride);
  w.slots = (__nv_bfloat16*)take(2 * w.ns * w.astride * (size_t)w.nslots);
  for (int q = 0; q < 5; ++q) {
    float* m = (float*)take(sizeof(float) * 2 * plane);
    w.f[q] = Master{m, m ? m + plane : nullptr};
  }
  const size_t stacked = (size_t)L * w.ncp * w.ldm;
  float* bb = (float*)take(sizeof(float) * 2 * stacked);
  w.bbar = Master{bb, bb ? bb + stacked : nullptr};
  w.ck_base = (float*)take(sizeof(float) * 2 * plane * (size_t)w.nseg);
  w.partial = (double2*)take(sizeof(double2) * (size_t)(L + 1) * w.ncta);
  w.flags = (unsigned int*)take(sizeof(unsigned int) * CHAIN_MAXP * (size_t)(w.ncp / BM));
  w.tau_partial = (double2*)take(sizeof(double2) * n);
  w.tau = (double2*)take(sizeof(double2));
  if (out) *out = w;
  return off;
}

// One split GEMM Y = left . right^T (right real) with epilogue EPI, for the plan's slice count
// and tile width.
struct GemmCtx {
  int n, np, kp, ncp, ns, bn;
  size_t bstride, astride;
};

// Left operand: `rows` rows of kp BF16 per slice (a multiple of 128), slice q at left + q * lstride.
struct Left {
  const __nv_bfloat16* base;
  size_t lstride;
  int rows;
};

template <int NS, int BN, int BKE, int EPI>
fq_status gemm_cfg(const GemmCtx& c, Left left, const __nv_bfloat16* right, const SplitEpi& e, cudaStream_t s) {
  using Cfg = SplitCfg<NS, BN, BKE, false>;
  SplitMaps maps{};
  fq_status st;
  for (int q = 0; q < NS; ++q) {
    if ((st = make_map(&maps.a[q], left.base + q * left.lstride, left.rows, c.kp, BM, BKE)) != FQ_OK) return st;
    if ((st = make_map(&maps.os[q], right + q * c.bstride, c.np, c.np, BN, BKE)) != FQ_OK) return st;
  }
  // the forward and adjoint terms run persistently (epilogue overlapped with the next tile's
  // MMAs); the gradient dot keeps one tile per CTA for its per-CTA partial sums
  constexpr bool persist = EPI != EPI_DOT;
  static std::atomic<unsigned> attr_set{0};
  if (fq_first_on_device(attr_set)) {
    cudaError_t r;
    if constexpr (persist)
      r = cudaFuncSetAttribute(k_split_persist<NS, BN, BKE, EPI, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)Cfg::SMEM);
    else
      r = cudaFuncSetAttribute(k_split_term<NS, BN, BKE, EPI, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)Cfg::SMEM);
    if (r != cudaSuccess) return fq_cuda_fail(r, "split gradient kernel shared-memory attribute");
  }
  const int sms = fq_sm_count();
  const int tiles_i = c.np / BN, tiles_j = left.rows / BM, nk = c.np / BKE;
  if constexpr (persist)
    k_split_persist<NS, BN, BKE, EPI, false><<<std::min(tiles_i * tiles_j, sms), PTHREADS, Cfg::SMEM, s>>>(
        maps, nk, tiles_j, tiles_i, e);
  else
    k_split_term<NS, BN, BKE, EPI, false><<<tiles_i * tiles_j, NTHREADS, Cfg::SMEM, s>>>(maps, nk, tiles_j, tiles_i,
                                                                                        e);
  return FQ_OK;
}

template <int EPI>
fq_status gemm(const GemmCtx& c, Left left, const __nv_bfloat16* right, const SplitEpi& e, cudaStream_t s) {
  if (c.ns == 3)
    return c.bn == 128 ? gemm_cfg<3, 128, 32, EPI>(c, left, right, e, s) : gemm_cfg<3, 64, 32, EPI>(c, left, right, e, s);
  return c.bn == 128 ? gemm_cfg<2, 128, 32, EPI>(c, left, right, e, s) : gemm_cfg<2, 64, 64, EPI>(c, left, right, e, s);
}

// A chain of products with one right operand (the step's Omega~_m) as one cooperative launch
// (split_core.cuh); FQ_EUNSUPPORTED where a chain cannot run (the caller launches each product).
template <int NS, int BN, int BKE, int EPI>
fq_status chain_cfg(const GemmCtx& c, const Left* lefts, const SplitEpi* eps, int nprod, const __nv_bfloat16* right,
                    unsigned int* flags, cudaStream_t s) {
  if (nprod > CHAIN_MAXP) return FQ_EUNSUPPORTED;
  ChainArgs ch{};
  fq_status st;
  for (int q = 0; q < NS; ++q)
    if ((st = make_map(&ch.rmaps.os[q], right + q * c.bstride, c.np, c.np, BN, BKE)) != FQ_OK) return st;
  for (int pp = 0; pp < nprod; ++pp) {
    for (int q = 0; q < NS; ++q)
      if ((st = make_map(&ch.left[pp][q], lefts[pp].base + q * lefts[pp].lstride, lefts[pp].rows, c.kp, BM, BKE)) !=
          FQ_OK)
        return st;
    ch.epi[pp] = eps[pp];
  }
  ch.nprod = nprod;
  ch.nk = c.np / BKE;
  ch.tiles_i = c.np / BN;
  ch.tiles_j = lefts[0].rows / BM;
  ch.flags = flags;
  cudaError_t ce = cudaMemsetAsync(flags, 0, sizeof(unsigned int) * (size_t)nprod * ch.tiles_j, s);
  if (ce != cudaSuccess) return fq_cuda_fail(ce, "chain counters");
  return launch_chain<NS, BN, BKE, EPI, false>(ch, s);
}

template <int EPI>
fq_status chain(const GemmCtx& c, const Left* lefts, const SplitEpi* eps, int nprod, const __nv_bfloat16* right,
                unsigned int* flags, cudaStream_t s) {
  if (c.ns == 3)
    return c.bn == 128 ? chain_cfg<3, 128, 32, EPI>(c, lefts, eps, nprod, right, flags, s)
                       : chain_cfg<3, 64, 32, EPI>(c, lefts, eps, nprod, right, flags, s);
  return c.bn == 128 ? chain_cfg<2, 128, 32, EPI>(c, lefts, eps, nprod, right, flags, s)
                     : chain_cfg<2, 64, 64, EPI>(c, lefts, eps, nprod, right, flags, s);
}

// The products of a chain: one cooperative launch, else one launch each.
template <int EPI>
fq_status run_products(const GemmCtx& c, const std::vector<Left>& lefts, const std::vector<SplitEpi>& eps,
                       const __nv_bfloat16* right, unsigned int* flags, cudaStream_t s) {
  const int nprod = (int)eps.size();
  fq_status st = chain<EPI>(c, lefts.data(), eps.data(), nprod, right, flags, s);
  if (st != FQ_EUNSUPPORTED) return st;
  for (int pp = 0; pp < nprod; ++pp)
    if ((st = gemm<EPI>(c, lefts[pp], right, eps[pp], s)) != FQ_OK) return st;
  return FQ_OK;
}

template <int NS>
void launch_real_slices(const fq_plan* p, const double* f, int m, bool omega, const SplitGradWs& w, cudaStream_t s) {
  if (omega)
    k_real_slices<NS><<<grid_n(w.bstride), 256, 0, s>>>(p->d_h0, p->d_h1, f, m, 1.0 / p->delta_e, p->sbeta, p->n, w.np,
                                                         w.S, w.bstride);
  else
    k_real_slices<NS><<<grid_n(w.bstride), 256, 0, s>>>(nullptr, p->d_h1, nullptr, 0, 1.0 / p->delta_e, 0.0, p->n,
                                                         w.np, w.E, w.bstride);
}

template <int NS>
void launch_scale_slices(const SplitGradWs& w, int n, Master in, float cr, float ci, Master out, __nv_bfloat16* sl,
                         size_t stride, cudaStream_t s) {
  k_scale_slices<NS><<<grid_n((size_t)n * n), 256, 0, s>>>(in.re, in.im, cr, ci, out.re, out.im, n, n, w.ldm, w.np,
                                                            w.kp, sl, stride);
}

struct Runner {
  fq_plan* p;
  const double* f;
  SplitGradWs w;
  GemmCtx c;
  cudaStream_t s;

  void omega(int m) {
    if (w.ns == 3) launch_real_slices<3>(p, f, m, true, w, s);
    else launch_real_slices<2>(p, f, m, true, w, s);
  }
  void scale_slices(Master in, float cr, float ci, Master out, __nv_bfloat16* sl, size_t stride) {
    if (w.ns == 3) launch_scale_slices<3>(w, p->n, in, cr, ci, out, sl, stride, s);
    else launch_scale_slices<2>(w, p->n, in, cr, ci, out, sl, stride, s);
  }
  SplitEpi epi() const {
    SplitEpi e{};
    e.n = p->n;
    e.nc = p->n;
    e.ldm = w.ldm;
    e.np = w.np;
    e.kp = w.kp;
    e.slice_stride = w.astride;
    e.t.status = p->d_status;
    return e;
  }

  // Step m of the forward chain: X_{m-1} in master f[*xb] with slices left[0] -> X_m in a master
  // of f[0..2] (returned through xb) with slices left[L]; left[l] receives the slices of psi_l.
  // `stride`: elements between the slices of one left operand.
  fq_status step(int m, int* xb, __nv_bfloat16* const* left, size_t stride) {
    const int L = p->L;
    omega(m);
    fq_term t{};
    t.coef0 = p->cheb[0];
    t.ph_re = p->phase_re;
    t.ph_im = p->phase_im;
    t.bound2 = 1.0 + 2e-3;
    t.status = p->d_status;
    int cur = *xb, nxt = (*xb + 1) % 3, acc = (*xb + 2) % 3, prv = -1;
    std::vector<SplitEpi> eps(L);
    std::vector<Left> lefts(L);
    for (int l = 0; l < L; ++l) {
      t.first = l == 0;
      t.last = l == L - 1;
      t.coef = p->cheb[l + 1];
      const int out = l == 0 ? nxt : prv;
      SplitEpi e = epi();
      e.cur_re = w.f[cur].re;
      e.cur_im = w.f[cur].im;
      e.prev_re = prv >= 0 ? w.f[prv].re : w.f[cur].re;
      e.prev_im = prv >= 0 ? w.f[prv].im : w.f[cur].im;
      e.acc_re = w.f[acc].re;
      e.acc_im = w.f[acc].im;
      e.out_re = w.f[out].re;
      e.out_im = w.f[out].im;
      e.slice_out = left[l + 1];
      e.slice_stride = stride;
      e.t = t;
      eps[l] = e;
      lefts[l] = Left{left[l], stride, w.ncp};
      if (t.last) {
        *xb = out;
      } else {
        prv = cur;
        cur = out;
      }
    }
    return run_products<EPI_FWD>(c, lefts, eps, w.S, w.flags, s);
  }
};

}  // namespace

size_t fq_grad_split_workspace(const fq_plan* p) { return split_grad_layout(p, nullptr, nullptr); }

fq_status fq_grad_split(fq_plan* p, const double* d_f, const void* d_W, double* d_loss, double* d_grad, void* d_ws,
                        cudaStream_t s) {
  fq_status st = encode_fn();
  if (st != FQ_OK) return st;
  Runner r{};
  r.p = p;
  r.f = d_f;
  r.s = s;
  split_grad_layout(p, d_ws, &r.w);
  SplitGradWs& w = r.w;
  r.c = GemmCtx{p->n, w.np, w.kp, w.ncp, w.ns, p->tile_n == 128 ? 128 : 64, w.bstride, w.astride};
  const int n = p->n, M = p->steps, L = p->L, S = p->stride;
  const size_t plane_bytes = sizeof(float) * (size_t)n * w.ldm;

  // slices and bbar are written only inside N x N: zero them once (padding rows and columns)
  cudaMemsetAsync(w.lsl[0], 0, sizeof(__nv_bfloat16) * w.ns * w.astride, s);
  cudaMemsetAsync(w.lsl[1], 0, sizeof(__nv_bfloat16) * w.ns * w.astride, s);
  cudaMemsetAsync(w.slots, 0, sizeof(__nv_bfloat16) * w.ns * w.astride * (size_t)w.nslots, s);
  cudaMemsetAsync(w.bbar.re, 0, sizeof(float) * 2 * (size_t)L * w.ncp * w.ldm, s);
  if (w.ns == 3) launch_real_slices<3>(p, nullptr, 0, false, w, s);
  else launch_real_slices<2>(p, nullptr, 0, false, w, s);

  // ---- forward sweep, checkpoints X_{kS} as FP32 masters
  int xb = 0;
  r.scale_slices(Master{nullptr, nullptr}, 1.f, 0.f, w.f[0], w.lsl[0], w.astride);
  cudaMemcpyAsync(w.ckpt(0, n).re, w.f[0].re, 2 * plane_bytes, cudaMemcpyDeviceToDevice, s);
  std::vector<__nv_bfloat16*> left(L + 1);
  for (int m = 0; m < M; ++m) {
    for (int l = 0; l <= L; ++l) left[l] = w.lsl[l & 1];
    if ((st = r.step(m, &xb, left.data(), w.astride)) != FQ_OK) return st;
    // the last term wrote X_m's slices into left[L]; the next step reads them from lsl[0]
    if (L & 1) std::swap(w.lsl[0], w.lsl[1]);
    if ((m + 1) % S == 0 && (m + 1) / S < w.nseg)
      cudaMemcpyAsync(w.ckpt((m + 1) / S, n).re, w.f[xb].re, 2 * plane_bytes, cudaMemcpyDeviceToDevice, s);
  }
  // ---- loss and seed
  k_trace_f32<<<n, 256, 0, s>>>((const double2*)d_W, w.f[xb].re, w.f[xb].im, n, w.ldm, w.tau_partial);
  fq_launch_loss(w.tau_partial, n, n, d_loss, w.tau, s);
  int gi = 3, gn = 4;  // G of the current step, and the buffer that receives bbar_0 = G_{m-1}
  k_seed_f32<<<grid_n((size_t)n * n), 256, 0, s>>>((const double2*)d_W, w.tau, n, w.ldm, w.f[gi].re, w.f[gi].im);

  // ---- backward, one checkpoint segment at a time
  const float cph_r = (float)p->phase_re, cph_i = (float)-p->phase_im;  // conj(e^{-i beta h})
  const size_t ss = w.slot_slice();
  for (int k = w.nseg - 1; k >= 0; --k) {
    const int m0 = k * S, m1 = std::min(M, m0 + S);
    // recompute the segment forward keeping the slices of every psi_l (slot st * L + l)
    cudaMemcpyAsync(w.f[0].re, w.ckpt(k, n).re, 2 * plane_bytes, cudaMemcpyDeviceToDevice, s);
    r.scale_slices(w.f[0], 1.f, 0.f, Master{nullptr, nullptr}, w.slot(0), ss);
    xb = 0;
    for (int st_ = 0; st_ < m1 - m0; ++st_) {
      for (int l = 0; l <= L; ++l) left[l] = w.slot(st_ * L + l);
      if ((st = r.step(m0 + st_, &xb, left.data(), ss)) != FQ_OK) return st;
    }
    for (int st_ = m1 - m0 - 1; st_ >= 0; --st_) {
      const int m = m0 + st_;
      r.omega(m);
      // bbar_L = conj(phase) a_L G (FP32 in its stacked block, slices in lsl[0])
      const double aL = p->cheb[L];
      r.scale_slices(w.f[gi], (float)(cph_r * aL), (float)(cph_i * aL), w.bbar_block(L), w.lsl[0], w.astride);
      int sl = 0;
      std::vector<SplitEpi> aeps;
      std::vector<Left> alefts;
      for (int l = L - 1; l >= 0; --l) {
        const double a = p->cheb[l];
        const Master out = l >= 1 ? w.bbar_block(l) : w.f[gn];
        SplitEpi e = r.epi();
        e.cur_re = w.f[gi].re;
        e.cur_im = w.f[gi].im;
        e.prev_re = l + 2 <= L ? w.bbar_block(l + 2).re : nullptr;
        e.prev_im = l + 2 <= L ? w.bbar_block(l + 2).im : nullptr;
        e.out_re = out.re;
        e.out_im = out.im;
        e.slice_out = w.lsl[sl ^ 1];
        e.cpa_re = (float)(cph_r * a);
        e.cpa_im = (float)(cph_i * a);
        e.cw = l == 0 ? 1.f : 2.f;
        e.t.bound2 = 1e30;  // NaN / overflow check only
        aeps.push_back(e);
        alefts.push_back(Left{w.lsl[sl], w.astride, w.ncp});
        sl ^= 1;
      }
      if ((st = run_products<EPI_ADJ>(r.c, alefts, aeps, w.S, w.flags, s)) != FQ_OK) return st;
      // D_l = <bbar_l, E psi_{l-1}>, l = 1..L, as one GEMM over the L stacked blocks: psi_0..psi_{L-1}
      // are the consecutive slots st*L .. st*L+L-1, bbar_1..bbar_L the stacked FP32 blocks
      SplitEpi d = r.epi();
      d.nc = L * w.ncp;
      d.cur_re = w.bbar.re;
      d.cur_im = w.bbar.im;
      d.partial = w.partial + w.ncta;  // block l at partial + l * ncta
      if ((st = gemm<EPI_DOT>(r.c, Left{w.slot(st_ * L), ss, L * w.ncp}, w.E, d, s)) != FQ_OK) return st;
      fq_launch_grad_reduce(w.partial, w.ncta, L, d_grad + m, s);
      std::swap(gi, gn);  // bbar_0 is the next G
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fq_cuda_fail(e, "split gradient kernels");
  return FQ_OK;
}
