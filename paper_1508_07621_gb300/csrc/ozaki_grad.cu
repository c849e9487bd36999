// floquet_grad in FP64 emulation (FQ_OZAKI plans): the reverse-mode chain of adjoint.cu (loss
// L = 1 - |Tr(W^+ U_T)|^2 / N^2, Clenshaw-form adjoint of Eqs. 10 and 12, dL/df_m from the kept
// forward Chebyshev vectors) with every N x N x N product on the tensor cores through the
// fixed-point slices of ozaki_core.cuh, FP64 states and FP64 epilogues.
//
// Piecewise-constant f makes Omega~_m = (H0 + f_m H1 - beta) / Delta E real symmetric, so every
// product has a real right operand (k_oz_real_term of ozaki_real.cuh: the real and imaginary rows
// of 64 states stacked as one 128-row MMA operand, double-buffered drains):
//   forward term   (OZ_FWD): psi_{l+1} = -2i Y + psi_{l-1}, acc += a_{l+1} psi_{l+1}, phase;
//   adjoint term   (OZ_ADJ): bbar_l = conj(e^{-i beta h}) a_l G + i cw Omega~ bbar_{l+1} + bbar_{l+2}
//                            (cw = 2, and 1 for l = 0);
//   gradient dot   (OZ_DOT): D_l = <bbar_l, E psi_{l-1}> with E = H1 / Delta E, per-CTA partials;
//   dL/df_m = 2 Re sum_l w_l D_l  (w_1 = -i, w_l = -2i).
// Every product's output is sliced again by k_oz_slice_left (row scales need whole rows).
// Memory: FP64 checkpoints of X every s = checkpoint_stride steps; each segment is recomputed
// once with the slices of every psi_l kept (the left operands of the dot products), slice-major
// ([slice][slot][row][k]) so that the L dots of a step run as one product over L x Np stacked
// rows against the stacked FP64 bbar_1 .. bbar_L.
#include <vector>

#include "ozaki_real.cuh"

namespace {

struct Planes {
  double* re;
  double* im;
};

struct OzGradWs {
  int np, ncp, nseg, nslots, ncta;
  size_t astride, rstride, plane;
  __nv_bfloat16* S;       // slices of Omega~_m
  int* etS;
  __nv_bfloat16* E;       // slices of E = H1 / Delta E
  int* etE;
  __nv_bfloat16* lsl[2];  // left-operand ping-pong (forward sweep, adjoint terms)
  int* esl[2];
  __nv_bfloat16* slots;   // psi_l slices of one recomputed segment: OZ_S x nslots x [ncp][2 np]
  int* es_slots;          // [nslots][ncp]
  Planes f[5];            // FP64 states [n][n]: forward cur / prev / acc; adjoint G and the next G
  Planes bbar;            // bbar_1 .. bbar_L of one step: L blocks of [ncp][n] (padding rows zero)
  double* ck_base;        // nseg checkpoints of X, each 2 planes [n][n]
  double2* partial;       // (L + 1) x ncta
  double2* tau_partial;   // n
  double2* tau;
  size_t slot_slice() const { return (size_t)nslots * astride; }
  __nv_bfloat16* slot(int q) const { return slots + (size_t)q * astride; }
  int* es_slot(int q) const { return es_slots + (size_t)q * ncp; }
  Planes bbar_block(int l, int n) const {  // bbar_l, l = 1..L
    const size_t o = (size_t)(l - 1) * ncp * n;
    return Planes{bbar.re + o, bbar.im + o};
  }
  Planes ckpt(int k) const {
    double* b = ck_base + (size_t)k * 2 * plane;
    return Planes{b, b + plane};
  }
};

size_t up(size_t x) { return (x + 255) & ~(size_t)255; }

size_t oz_grad_layout(const fq_plan* p, void* base, OzGradWs* out) {
  OzGradWs w{};
  const int n = p->n, L = p->L, s = p->stride;
  w.np = (n + 127) & ~127;
  w.ncp = w.np;
  w.nseg = (p->steps + s - 1) / s;
  w.nslots = s * L + 1;
  w.astride = (size_t)w.ncp * 2 * w.np;
  w.rstride = (size_t)w.np * w.np;
  w.plane = (size_t)n * n;
  w.ncta = (w.ncp / OZR_BM) * (w.np / OZ_BN);
  char* b = (char*)base;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* q = b ? b + off : nullptr;
    off += up(bytes);
    return q;
  };
  const size_t bf = sizeof(__nv_bfloat16);
  w.S = (__nv_bfloat16*)take(bf * OZ_S * w.rstride);
  w.etS = (int*)take(sizeof(int) * w.np);
  w.E = (__nv_bfloat16*)take(bf * OZ_S * w.rstride);
  w.etE = (int*)take(sizeof(int) * w.np);
  for (int q = 0; q < 2; ++q) {
    w.lsl[q] = (__nv_bfloat16*)take(bf * OZ_S * w.astride);
    w.esl[q] = (int*)take(sizeof(int) * w.ncp);
  }
  w.slots = (__nv_bfloat16*)take(bf * OZ_S * w.astride * (size_t)w.nslots);
  w.es_slots = (int*)take(sizeof(int) * w.ncp * (size_t)w.nslots);
  for (int q = 0; q < 5; ++q) {
    double* m = (double*)take(sizeof(double) * 2 * w.plane);
    w.f[q] = Planes{m, m ? m + w.plane : nullptr};
  }
  const size_t stacked = (size_t)L * w.ncp * n;
  double* bb = (double*)take(sizeof(double) * 2 * stacked);
  w.bbar = Planes{bb, bb ? bb + stacked : nullptr};
  w.ck_base = (double*)take(sizeof(double) * 2 * w.plane * (size_t)w.nseg);
  w.partial = (double2*)take(sizeof(double2) * (size_t)(L + 1) * w.ncta);
  w.tau_partial = (double2*)take(sizeof(double2) * n);
  w.tau = (double2*)take(sizeof(double2));
  if (out) *out = w;
  return off;
}

// One product Y = left . right^T (right real, [np][np] slices) with epilogue EPI over `rows` left rows.
template <int EPI>
fq_status oz_gemm(const OzGradWs& w, const __nv_bfloat16* left, size_t lstride, int rows, const __nv_bfloat16* right,
                  const OzEpi& e, cudaStream_t s) {
  OzMaps maps{};
  fq_status st;
  for (int q = 0; q < OZ_S; ++q) {
    if ((st = make_map(&maps.a[q], left + q * lstride, rows, 2 * w.np, OZR_BM, OZ_BKE)) != FQ_OK) return st;
    if ((st = make_map(&maps.r[q], right + q * w.rstride, w.np, w.np, OZ_BN, OZ_BKE)) != FQ_OK) return st;
  }
  static std::atomic<unsigned> attr_set{0};
  if (fq_first_on_device(attr_set)) {
    cudaError_t r = cudaFuncSetAttribute(k_oz_real_term<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)OZR_SMEM);
    if (r != cudaSuccess) return fq_cuda_fail(r, "FP64-emulation gradient kernel shared-memory attribute");
  }
  const int tiles_i = w.np / OZ_BN, tiles_j = rows / OZR_BM;
  k_oz_real_term<EPI><<<tiles_i * tiles_j, OZ_THREADS, OZR_SMEM, s>>>(maps, w.np / OZ_BKE, tiles_j, tiles_i, w.np, e);
  return FQ_OK;
}

struct Runner {
  fq_plan* p;
  const double* f;
  OzGradWs w;
  cudaStream_t s;

  void omega(int m) {
    k_oz_real<<<w.np, 256, 0, s>>>(p->d_h0, p->d_h1, f, m, 1.0 / p->delta_e, p->sbeta, p->n, w.np, w.rstride, w.S,
                                   w.etS);
  }
  // slices of v = c x (x NULL: identity rows) into `left` (slice stride lstride) and es; FP64
  // copy of v into `out` when given
  void slice(Planes x, double cr, double ci, Planes out, __nv_bfloat16* left, size_t lstride, int* es) {
    k_oz_slice_left<<<w.ncp, 256, 0, s>>>(x.re, x.im, cr, ci, out.re, out.im, p->n, p->n, w.np, lstride, left, es);
  }
  OzEpi epi() const {
    OzEpi e{};
    e.n = p->n;
    e.nc = p->n;
    e.t.status = p->d_status;
    return e;
  }

  // Step m of the forward chain: X_{m-1} in f[*xb] with slices left[0] -> X_m in one of f[0..2]
  // (returned through xb) with slices left[L]; left[l] receives the slices of psi_l.
  fq_status step(int m, int* xb, __nv_bfloat16* const* left, int* const* es, size_t lstride) {
    const int L = p->L;
    omega(m);
    fq_term t{};
    t.coef0 = p->cheb[0];
    t.ph_re = p->phase_re;
    t.ph_im = p->phase_im;
    t.bound2 = 1.0 + 1e-9;
    t.status = p->d_status;
    int cur = *xb, nxt = (*xb + 1) % 3, acc = (*xb + 2) % 3, prv = -1;
    for (int l = 0; l < L; ++l) {
      t.first = l == 0;
      t.last = l == L - 1;
      t.coef = p->cheb[l + 1];
      const int out = l == 0 ? nxt : prv;
      OzEpi e = epi();
      e.cur_re = w.f[cur].re;
      e.cur_im = w.f[cur].im;
      e.prev_re = prv >= 0 ? w.f[prv].re : w.f[cur].re;
      e.prev_im = prv >= 0 ? w.f[prv].im : w.f[cur].im;
      e.acc_re = w.f[acc].re;
      e.acc_im = w.f[acc].im;
      e.out_re = w.f[out].re;
      e.out_im = w.f[out].im;
      e.es = es[l];
      e.et = w.etS;
      e.t = t;
      fq_status st = oz_gemm<OZ_FWD>(w, left[l], lstride, w.ncp, w.S, e, s);
      if (st != FQ_OK) return st;
      slice(w.f[out], 1.0, 0.0, Planes{nullptr, nullptr}, left[l + 1], lstride, es[l + 1]);
      if (t.last) {
        *xb = out;
      } else {
        prv = cur;
        cur = out;
      }
    }
    return FQ_OK;
  }
};

}  // namespace

size_t fq_grad_ozaki_workspace(const fq_plan* p) { return oz_grad_layout(p, nullptr, nullptr); }

fq_status fq_grad_ozaki(fq_plan* p, const double* d_f, const void* d_W, double* d_loss, double* d_grad, void* d_ws,
                        cudaStream_t s) {
  fq_status st = encode_fn();
  if (st != FQ_OK) return st;
  Runner r{};
  r.p = p;
  r.f = d_f;
  r.s = s;
  oz_grad_layout(p, d_ws, &r.w);
  OzGradWs& w = r.w;
  const int n = p->n, M = p->steps, L = p->L, S = p->stride;
  const size_t plane2 = 2 * sizeof(double) * w.plane;

  // the stacked bbar blocks are written only in their first n rows: zero the padding once
  cudaMemsetAsync(w.bbar.re, 0, sizeof(double) * 2 * (size_t)L * w.ncp * n, s);
  k_oz_real<<<w.np, 256, 0, s>>>(nullptr, p->d_h1, nullptr, 0, 1.0 / p->delta_e, 0.0, n, w.np, w.rstride, w.E, w.etE);

  // ---- forward sweep, checkpoints X_{kS}
  int xb = 0;
  r.slice(Planes{nullptr, nullptr}, 1.0, 0.0, w.f[0], w.lsl[0], w.astride, w.esl[0]);
  cudaMemcpyAsync(w.ckpt(0).re, w.f[0].re, plane2, cudaMemcpyDeviceToDevice, s);
  std::vector<__nv_bfloat16*> left(L + 1);
  std::vector<int*> es(L + 1);
  for (int m = 0; m < M; ++m) {
    for (int l = 0; l <= L; ++l) {
      left[l] = w.lsl[l & 1];
      es[l] = w.esl[l & 1];
    }
    if ((st = r.step(m, &xb, left.data(), es.data(), w.astride)) != FQ_OK) return st;
    // the last term's slices are in left[L]; the next step reads them from lsl[0]
    if (L & 1) {
      std::swap(w.lsl[0], w.lsl[1]);
      std::swap(w.esl[0], w.esl[1]);
    }
    if ((m + 1) % S == 0 && (m + 1) / S < w.nseg)
      cudaMemcpyAsync(w.ckpt((m + 1) / S).re, w.f[xb].re, plane2, cudaMemcpyDeviceToDevice, s);
  }
  // ---- loss and seed
  fq_launch_trace_f64((const double*)d_W, w.f[xb].re, w.f[xb].im, n, w.tau_partial, s);
  fq_launch_loss(w.tau_partial, n, n, d_loss, w.tau, s);
  int gi = 3, gn = 4;  // G of the current step, and the buffer that receives bbar_0 = G_{m-1}
  fq_launch_seed_f64((const double*)d_W, w.tau, n, w.f[gi].re, w.f[gi].im, s);

  // ---- backward, one checkpoint segment at a time
  const double cph_r = p->phase_re, cph_i = -p->phase_im;  // conj(e^{-i beta h})
  const size_t ss = w.slot_slice();
  for (int k = w.nseg - 1; k >= 0; --k) {
    const int m0 = k * S, m1 = std::min(M, m0 + S);
    // recompute the segment forward keeping the slices of every psi_l (slot st * L + l)
    cudaMemcpyAsync(w.f[0].re, w.ckpt(k).re, plane2, cudaMemcpyDeviceToDevice, s);
    r.slice(w.f[0], 1.0, 0.0, Planes{nullptr, nullptr}, w.slot(0), ss, w.es_slot(0));
    xb = 0;
    for (int st_ = 0; st_ < m1 - m0; ++st_) {
      for (int l = 0; l <= L; ++l) {
        left[l] = w.slot(st_ * L + l);
        es[l] = w.es_slot(st_ * L + l);
      }
      if ((st = r.step(m0 + st_, &xb, left.data(), es.data(), ss)) != FQ_OK) return st;
    }
    for (int st_ = m1 - m0 - 1; st_ >= 0; --st_) {
      const int m = m0 + st_;
      r.omega(m);
      // bbar_L = conj(phase) a_L G (FP64 in its stacked block, slices in lsl[0])
      const double aL = p->cheb[L];
      r.slice(w.f[gi], cph_r * aL, cph_i * aL, w.bbar_block(L, n), w.lsl[0], w.astride, w.esl[0]);
      int sl = 0;
      for (int l = L - 1; l >= 0; --l) {
        const double a = p->cheb[l];
        const Planes out = l >= 1 ? w.bbar_block(l, n) : w.f[gn];
        OzEpi e = r.epi();
        e.cur_re = w.f[gi].re;
        e.cur_im = w.f[gi].im;
        e.prev_re = l + 2 <= L ? w.bbar_block(l + 2, n).re : nullptr;
        e.prev_im = l + 2 <= L ? w.bbar_block(l + 2, n).im : nullptr;
        e.out_re = out.re;
        e.out_im = out.im;
        e.es = w.esl[sl];
        e.et = w.etS;
        e.cpa_re = cph_r * a;
        e.cpa_im = cph_i * a;
        e.cw = l == 0 ? 1.0 : 2.0;
        e.t.bound2 = 1e300;  // NaN / overflow check only
        if ((st = oz_gemm<OZ_ADJ>(w, w.lsl[sl], w.astride, w.ncp, w.S, e, s)) != FQ_OK) return st;
        if (l >= 1) r.slice(out, 1.0, 0.0, Planes{nullptr, nullptr}, w.lsl[sl ^ 1], w.astride, w.esl[sl ^ 1]);
        sl ^= 1;
      }
      // D_l = <bbar_l, E psi_{l-1}>, l = 1..L, as one product over the L stacked blocks:
      // psi_0..psi_{L-1} are the consecutive slots st*L .. st*L+L-1, bbar_1..bbar_L the stacked blocks
      OzEpi d = r.epi();
      d.nc = L * w.ncp;
      d.cur_re = w.bbar.re;
      d.cur_im = w.bbar.im;
      d.es = w.es_slot(st_ * L);
      d.et = w.etE;
      d.partial = w.partial + w.ncta;  // block l at partial + l * ncta
      if ((st = oz_gemm<OZ_DOT>(w, w.slot(st_ * L), ss, L * w.ncp, w.E, d, s)) != FQ_OK) return st;
      fq_launch_grad_reduce(w.partial, w.ncta, L, d_grad + m, s);
      std::swap(gi, gn);  // bbar_0 is the next G
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fq_cuda_fail(e, "FP64-emulation gradient kernels");
  return FQ_OK;
}
