// C ABI: plan lifetime, workspace layout and the host loops that chain the kernels
// (the propagation part of Algorithm 1: M steps of L Chebyshev terms each, U_T written in place).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "internal.h"

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// Carves aligned regions out of the caller's workspace.
struct Carver {
  char* base;
  size_t used = 0;
  explicit Carver(void* b) : base((char*)b) {}
  template <typename T>
  T* take(size_t count) {
    T* p = base ? (T*)(base + used) : nullptr;
    used += align_up(count * sizeof(T));
    return p;
  }
};

int tri_ld(int n) { return (n + 3) & ~3; }

// Workspace regions of floquet_propagate / floquet_build_UT.
struct StateWs {
  // dense FP64
  double* S = nullptr;
  double* A = nullptr;
  // tridiagonal coefficients [nsteps][ld] (d, er, ei contiguous)
  void* coeff = nullptr;
  // three planar state buffers
  void* buf[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
};

size_t layout(const fq_plan* p, int nc, int nsteps, void* ws, StateWs* out) {
  Carver c(ws);
  StateWs w;
  const int n = p->n;
  if (p->path == PATH_DENSE_F64 && p->dense_resident) {
    // Omega~ of a chunk of steps, one state block updated in place
    w.S = c.take<double>(fq_dense_resident_omega_count(n, nsteps));
    w.A = c.take<double>(fq_dense_resident_omega_count(n, nsteps));
    for (int q = 0; q < 2; ++q) w.buf[0][q] = c.take<double>((size_t)nc * n);
  } else if (p->path == PATH_DENSE_F64) {
    w.S = c.take<double>((size_t)n * n);
    w.A = c.take<double>((size_t)n * n);
    for (int b = 0; b < 3; ++b)
      for (int q = 0; q < 2; ++q) w.buf[b][q] = c.take<double>((size_t)nc * n);
  } else if (p->path == PATH_TRI_STREAM) {
    const size_t ld = tri_ld(n);
    const size_t es = p->precision == FQ_FP64 ? sizeof(double) : sizeof(float);
    w.coeff = c.take<char>(3 * ld * (size_t)nsteps * es);
    for (int b = 0; b < 3; ++b)
      for (int q = 0; q < 2; ++q) w.buf[b][q] = c.take<char>((size_t)nc * ld * es);
  } else if (p->path == PATH_TRI6) {
    const size_t ld = tri_ld(n);
    w.S = c.take<double>(7 * ld);  // Omega~_m's diagonals, re
    w.A = c.take<double>(7 * ld);  // and im
    for (int b = 0; b < 3; ++b)
      for (int q = 0; q < 2; ++q) w.buf[b][q] = c.take<double>((size_t)nc * ld);
  } else if (p->path == PATH_TRI_RESIDENT) {
    w.coeff = c.take<char>(fq_resident_coeff_bytes(n, nsteps));
  } else if (p->path == PATH_TRI_TILE) {
    w.coeff = c.take<char>(fq_tile_workspace(p, nc, nsteps));
  } else if (p->path == PATH_TRI_BAND) {
    w.coeff = c.take<char>(fq_band_workspace(p, nc, nsteps));
  } else if (p->path == PATH_DENSE_SPLIT) {
    w.coeff = c.take<char>(fq_split_workspace(p, nc, nullptr, nullptr));
  } else if (p->path == PATH_DENSE_OZAKI) {
    w.coeff = c.take<char>(fq_ozaki_workspace(p, nc, nullptr, nullptr));
  }
  if (out) *out = w;
  return c.used;
}

fq_status cuda_ok(cudaError_t e, const char* what) { return e == cudaSuccess ? FQ_OK : fq_cuda_fail(e, what); }

template <typename T>
fq_blk<T> blk(void* const (&b)[2]) { return fq_blk<T>{(T*)b[0], (T*)b[1]}; }

// Runs steps [m_begin, m_end) on the planar block held in buffer `x` (index into w.buf);
// returns the buffer index that holds the result.
template <typename T>
int run_chain(fq_plan* p, StateWs& w, int x, int nc, int m_begin, int m_end, cudaStream_t s) {
  const int n = p->n, L = p->L;
  const int ld = p->path == PATH_DENSE_F64 ? n : tri_ld(n);
  const int nsteps = m_end - m_begin;
  fq_term t{};
  t.coef0 = p->cheb[0];
  t.ph_re = p->phase_re;
  t.ph_im = p->phase_im;
  t.bound2 = p->precision == FQ_FP64 ? 1.0 + 1e-9 : 1.0 + 2e-3;
  t.status = p->d_status;
  const T* cd = nullptr;
  const T* cer = nullptr;
  const T* cei = nullptr;
  if (p->path == PATH_TRI_STREAM) {
    cd = (const T*)w.coeff;
    cer = cd + (size_t)nsteps * ld;
    cei = cer + (size_t)nsteps * ld;
  }
  for (int m = m_begin; m < m_end; ++m) {
    if (p->path == PATH_DENSE_F64 && p->order == 6) {
      double c[FQ_M6_TERMS];
      const double inv = 1.0 / (p->h * p->delta_e);
      for (int q = 0; q < FQ_M6_TERMS; ++q) c[q] = p->coef6[(size_t)m * FQ_M6_TERMS + q] * inv;
      fq_launch_omega6_f64(p, c, w.S, w.A, s);
    } else if (p->path == PATH_DENSE_F64) {
      fq_launch_omega_dense_f64(p->d_h0, p->d_h1, p->d_k, n, p->sa[m], p->sb[m], p->sc[m], p->sbeta, w.S, w.A, s);
    } else if (p->path == PATH_TRI6) {
      double c[FQ_M6_TERMS];
      const double inv = 1.0 / (p->h * p->delta_e);
      for (int q = 0; q < FQ_M6_TERMS; ++q) c[q] = p->coef6[(size_t)m * FQ_M6_TERMS + q] * inv;
      fq_launch_omega_band6(p, c, w.S, w.A, ld, s);
    }
    // buffers: cur = psi_l, prv = psi_{l-1}, acc; x holds psi_0
    int cur = x, nxt = (x + 1) % 3, acc = (x + 2) % 3;
    int prv = -1;
    for (int l = 0; l < L; ++l) {
      t.first = l == 0;
      t.last = l == L - 1;
      t.coef = p->cheb[l + 1];
      // output: psi_{l+1} goes to a fresh buffer on the first term, in place of psi_{l-1}
      // afterwards; the step result of a one-term step goes to the free third buffer
      const int out = l == 0 ? nxt : prv;
      const int pq = prv >= 0 ? prv : cur;  // psi_{l-1} (unused on the first term)
      if (p->path == PATH_DENSE_F64) {
        fq_launch_term_dense_f64(w.S, w.A, n, blk<double>(w.buf[cur]), blk<double>(w.buf[pq]),
                                 blk<double>(w.buf[acc]), blk<double>(w.buf[out]), nc, t, s);
      } else if (p->path == PATH_TRI6) {
        fq_launch_term_band6_f64(w.S, w.A, n, blk<double>(w.buf[cur]), blk<double>(w.buf[pq]),
                                 blk<double>(w.buf[acc]), blk<double>(w.buf[out]), nc, ld, t, s);
      } else {
        const size_t off = (size_t)(m - m_begin) * ld;
        if (sizeof(T) == 8)
          fq_launch_term_tri_f64((const double*)cd + off, (const double*)cer + off, (const double*)cei + off, n,
                                 blk<double>(w.buf[cur]), blk<double>(w.buf[pq]), blk<double>(w.buf[acc]),
                                 blk<double>(w.buf[out]), nc, ld, t, s);
        else
          fq_launch_term_tri_f32((const float*)cd + off, (const float*)cer + off, (const float*)cei + off, n,
                                 blk<float>(w.buf[cur]), blk<float>(w.buf[pq]), blk<float>(w.buf[acc]),
                                 blk<float>(w.buf[out]), nc, ld, t, s);
      }
      if (t.last) {
        x = out;
      } else {
        prv = cur;
        cur = out;
      }
    }
  }
  return x;
}

fq_status check_ws(const fq_plan* p, int nc, int nsteps, void* ws, size_t bytes) {
  const size_t need = layout(p, nc, nsteps, nullptr, nullptr);
  if (need > 0 && (!ws || bytes < need)) {
    fq_set_error("workspace too small: need %zu bytes, got %zu", need, bytes);
    return FQ_EINVAL;
  }
  if (ws && ((uintptr_t)ws & (kAlign - 1))) {
    fq_set_error("workspace must be 256-byte aligned");
    return FQ_EINVAL;
  }
  return FQ_OK;
}

fq_status propagate_impl(fq_plan* p, const double* x0, double* x, int nc, int m_begin, int m_end, int identity,
                         int transpose_out, void* ws, size_t ws_bytes, cudaStream_t s) {
  const int n = p->n;
  const int nsteps = m_end - m_begin;
  fq_status st = check_ws(p, nc, nsteps, ws, ws_bytes);
  if (st != FQ_OK) return st;
  if (nc == 0 || n == 0) return FQ_OK;
  StateWs w;
  layout(p, nc, nsteps, ws, &w);
  if (p->path == PATH_TRI_RESIDENT) {
    fq_launch_gauge_coeffs(p, m_begin, nsteps, w.coeff, s);
    st = fq_launch_resident(p, w.coeff, identity ? nullptr : x0, x, transpose_out, nc, m_begin, m_end, s);
    if (st != FQ_OK) return st;
    return cuda_ok(cudaGetLastError(), "resident chain");
  }
  if (p->path == PATH_TRI_TILE) {
    st = fq_tile_propagate(p, x0, x, nc, m_begin, m_end, identity, transpose_out, w.coeff, s);
    if (st != FQ_OK) return st;
    return cuda_ok(cudaGetLastError(), "tiled tridiagonal chain");
  }
  if (p->path == PATH_TRI_BAND) {
    st = fq_band_propagate(p, x0, x, nc, m_begin, m_end, identity, transpose_out, w.coeff, s);
    if (st != FQ_OK) return st;
    return cuda_ok(cudaGetLastError(), "band chain");
  }
  if (p->path == PATH_DENSE_SPLIT) {
    st = fq_split_propagate(p, x0, x, nc, m_begin, m_end, identity, transpose_out, w.coeff, s);
    if (st != FQ_OK) return st;
    return cuda_ok(cudaGetLastError(), "split-precision chain");
  }
  if (p->path == PATH_DENSE_OZAKI) {
    st = fq_ozaki_propagate(p, x0, x, nc, m_begin, m_end, identity, transpose_out, w.coeff, s);
    if (st != FQ_OK) return st;
    return cuda_ok(cudaGetLastError(), "FP64-emulation chain");
  }
  const bool f64 = p->precision == FQ_FP64 || p->path == PATH_DENSE_F64;  // dense FQ_DF32: FP64 states
  const int ld = p->path == PATH_DENSE_F64 ? n : tri_ld(n);
  if (p->path == PATH_TRI_STREAM) {
    if (f64) {
      double* d = (double*)w.coeff;
      fq_launch_tri_coeffs_f64(p, m_begin, nsteps, 1.0, d, d + (size_t)nsteps * ld, d + 2 * (size_t)nsteps * ld, s);
    } else {
      float* d = (float*)w.coeff;
      fq_launch_tri_coeffs_f32(p, m_begin, nsteps, 1.0, d, d + (size_t)nsteps * ld, d + 2 * (size_t)nsteps * ld, s);
    }
  }
  int xb = 0;
  if (f64) {
    fq_blk<double> b0 = blk<double>(w.buf[0]);
    if (identity) fq_launch_identity_f64(b0, nc, n, ld, s);
    else fq_launch_load_states(x0, b0, nc, n, ld, s);
    if (p->path == PATH_DENSE_F64 && p->dense_resident) {
      st = fq_dense_resident_chain(p, b0.re, b0.im, nc, m_begin, m_end, w.S, w.A, s);
      if (st != FQ_OK) return st;
    } else {
      xb = run_chain<double>(p, w, 0, nc, m_begin, m_end, s);
    }
    fq_blk<double> bx = blk<double>(w.buf[xb]);
    if (transpose_out) fq_launch_store_transpose_f64(bx, x, n, ld, s);
    else fq_launch_store_states_f64(bx, x, nc, n, ld, s);
  } else {
    fq_blk<float> b0 = blk<float>(w.buf[0]);
    if (identity) fq_launch_identity_f32(b0, nc, n, ld, s);
    else fq_launch_load_states_f32(x0, b0, nc, n, ld, s);
    xb = run_chain<float>(p, w, 0, nc, m_begin, m_end, s);
    fq_blk<float> bx = blk<float>(w.buf[xb]);
    if (transpose_out) fq_launch_store_transpose_f32(bx, x, n, ld, s);
    else fq_launch_store_states_f32(bx, x, nc, n, ld, s);
  }
  return cuda_ok(cudaGetLastError(), "propagation kernels");
}

void free_plan(fq_plan* p) {
  if (!p) return;
  for (void* d : {(void*)p->d_h0, (void*)p->d_h1, (void*)p->d_k, (void*)p->d_h0o, (void*)p->d_scal,
                  (void*)p->d_status, (void*)p->d_cm})
    if (d) cudaFree(d);
  if (p->ktimer) {
    for (cudaEvent_t e : p->ktimer->ev) cudaEventDestroy(e);
    delete p->ktimer;
  }
  delete p;
}

// Owns a plan under construction until it is handed to the caller.
struct PlanOwner {
  fq_plan* p;
  ~PlanOwner() { free_plan(p); }
  fq_plan* release() {
    fq_plan* q = p;
    p = nullptr;
    return q;
  }
};

fq_status plan_create(fq_plan** out, const fq_problem* prob) {
  PlanOwner own{new fq_plan()};  // frees the plan on every early return and on an exception
  fq_plan* p = own.p;
  // dense spectral bounds wait for H0, H1 on the device (their Lanczos products run there)
  fq_status st = fq_host_plan(prob, p, prob && prob->format == FQ_DENSE);
  if (st != FQ_OK) return st;
  const int n = p->n, M = p->steps;
  if (p->format == FQ_TRIDIAG && p->order == 6) {
    if (prob->kernel != FQ_KERNEL_AUTO && prob->kernel != FQ_KERNEL_STREAM) {
      fq_set_error("6th-order tridiagonal plans run on the streaming FP64 kernel");
      return FQ_EUNSUPPORTED;
    }
    p->path = PATH_TRI6;
  } else if (p->format == FQ_TRIDIAG) {
    const bool res_ok = p->precision == FQ_FP32 && fq_resident_supported(n, p->L);
    const bool tile_ok = fq_tile_supported(p->L) != 0;
    if (prob->kernel == FQ_KERNEL_RESIDENT && !res_ok) {
      fq_set_error("resident kernel needs FQ_FP32, N <= 10240 and L <= 128 (N = %d, L = %d)", n, p->L);
      return FQ_EUNSUPPORTED;
    }
    if ((prob->kernel == FQ_KERNEL_TILED || p->precision == FQ_DF32) && !tile_ok) {
      fq_set_error("tiled kernel needs L <= 128 (L = %d)", p->L);
      return FQ_EUNSUPPORTED;
    }
    if (p->precision == FQ_DF32 && prob->kernel != FQ_KERNEL_AUTO && prob->kernel != FQ_KERNEL_TILED) {
      fq_set_error("FQ_DF32 runs on the tiled kernel only");
      return FQ_EUNSUPPORTED;
    }
    if (p->precision == FQ_OZAKI || prob->kernel == FQ_KERNEL_BAND) {
      if (p->precision != FQ_OZAKI || (prob->kernel != FQ_KERNEL_AUTO && prob->kernel != FQ_KERNEL_BAND)) {
        fq_set_error("the band kernel runs FQ_OZAKI tridiagonal plans, and they run on it only");
        return FQ_EUNSUPPORTED;
      }
      if (!fq_band_supported(p->L)) {
        fq_set_error("band kernel needs L <= 47 (L = %d): more steps per period lower L", p->L);
        return FQ_EUNSUPPORTED;
      }
    }
    switch (prob->kernel) {
      case FQ_KERNEL_STREAM: p->path = PATH_TRI_STREAM; break;
      case FQ_KERNEL_RESIDENT: p->path = PATH_TRI_RESIDENT; break;
      case FQ_KERNEL_TILED: p->path = PATH_TRI_TILE; break;
      case FQ_KERNEL_BAND: p->path = PATH_TRI_BAND; break;
      default:
        p->path = p->precision == FQ_OZAKI ? PATH_TRI_BAND
                                           : (res_ok ? PATH_TRI_RESIDENT : (tile_ok ? PATH_TRI_TILE : PATH_TRI_STREAM));
    }
  } else {
    p->path = (p->precision == FQ_FP64 || p->precision == FQ_DF32)
                  ? PATH_DENSE_F64
                  : (p->precision == FQ_OZAKI ? PATH_DENSE_OZAKI : PATH_DENSE_SPLIT);
  }
  cudaGetDevice(&p->device);
  auto fail = [&](cudaError_t e, const char* what) {
    fq_status r = (e == cudaErrorMemoryAllocation) ? FQ_ENOMEM : FQ_ECUDA;
    fq_cuda_fail(e, what);
    return r;
  };
  cudaError_t e;
  const size_t opsz = p->format == FQ_DENSE ? (size_t)n * n : (size_t)n;
  if ((e = cudaMalloc(&p->d_h0, opsz * sizeof(double))) != cudaSuccess) return fail(e, "cudaMalloc H0");
  if ((e = cudaMalloc(&p->d_h1, opsz * sizeof(double))) != cudaSuccess) return fail(e, "cudaMalloc H1");
  if ((e = cudaMalloc(&p->d_k, std::max<size_t>(opsz, 1) * sizeof(double))) != cudaSuccess) return fail(e, "cudaMalloc K");
  if ((e = cudaMalloc(&p->d_scal, 3 * (size_t)M * sizeof(double))) != cudaSuccess) return fail(e, "cudaMalloc scalars");
  if ((e = cudaMalloc(&p->d_status, sizeof(unsigned int))) != cudaSuccess) return fail(e, "cudaMalloc status");
  if ((e = cudaMemset(p->d_status, 0, sizeof(unsigned int))) != cudaSuccess) return fail(e, "status clear");
  if ((e = cudaMemcpy(p->d_h0, prob->h0, opsz * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e, "upload H0");
  if ((e = cudaMemcpy(p->d_h1, prob->h1, opsz * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e, "upload H1");
  if (p->dense_bounds_pending) {
    // Lanczos on the device-resident H0, H1: each product reads the matrices at HBM rate, the
    // n-vectors travel over the link (reading R4)
    double *d_x = nullptr, *d_y = nullptr;
    if ((e = cudaMalloc(&d_x, 2 * (size_t)n * sizeof(double))) != cudaSuccess) return fail(e, "cudaMalloc Lanczos");
    d_y = d_x + n;
    cudaError_t ae = cudaSuccess;
    const fq_dense_apply apply = [&](int which, double g, const double* x, double* y) {
      if (ae != cudaSuccess) {
        std::fill(y, y + n, 0.0);
        return;
      }
      ae = cudaMemcpy(d_x, x, (size_t)n * sizeof(double), cudaMemcpyHostToDevice);
      if (ae == cudaSuccess) {
        fq_launch_symv2(p->d_h0, p->d_h1, g, which, d_x, d_y, n, 0);
        ae = cudaMemcpy(y, d_y, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost);
      }
      if (ae != cudaSuccess) std::fill(y, y + n, 0.0);
    };
    double emin, emax;
    fq_dense_bounds(n, p->dense_glo, p->dense_ghi, p->dense_kmax, apply, &emin, &emax);
    cudaFree(d_x);
    if (ae != cudaSuccess) return fail(ae, "Lanczos products");
    if ((st = fq_finish_computed_bounds(p, emin, emax)) != FQ_OK) return st;
    p->dense_bounds_pending = false;
  }
  std::vector<double> scal(3 * (size_t)M);
  std::copy(p->sa.begin(), p->sa.end(), scal.begin());
  std::copy(p->sb.begin(), p->sb.end(), scal.begin() + M);
  std::copy(p->sc.begin(), p->sc.end(), scal.begin() + 2 * M);
  if ((e = cudaMemcpy(p->d_scal, scal.data(), scal.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess)
    return fail(e, "upload scalars");
  if (p->format == FQ_DENSE) {
    // [H0, H1] = H0 H1 - H1 H0, once per plan (§3)
    fq_launch_gemm_f64(p->d_h0, p->d_h1, p->d_k, n, 1.0, 0.0, 0);
    fq_launch_gemm_f64(p->d_h1, p->d_h0, p->d_k, n, -1.0, 1.0, 0);
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(e, "commutator");
    if (p->order == 6) {
      // nested commutators K0 = [H0,K], K1 = [H1,K], K00 = [H0,K0], K01 = [H0,K1], K10 = [H1,K0],
      // K11 = [H1,K1], KK0 = [K,K0], KK1 = [K,K1], computed once (§3)
      const size_t nn = (size_t)n * n;
      if ((e = cudaMalloc(&p->d_cm, 8 * nn * sizeof(double))) != cudaSuccess) return fail(e, "cudaMalloc commutators");
      const double* K = p->d_k;
      double* C = p->d_cm;
      const double* lhs[8] = {p->d_h0, p->d_h1, p->d_h0, p->d_h0, p->d_h1, p->d_h1, K, K};
      const double* rhs[8] = {K, K, C + 0 * nn, C + 1 * nn, C + 0 * nn, C + 1 * nn, C + 0 * nn, C + 1 * nn};
      for (int q = 0; q < 8; ++q) {
        fq_launch_gemm_f64(lhs[q], rhs[q], C + q * nn, n, 1.0, 0.0, 0);
        fq_launch_gemm_f64(rhs[q], lhs[q], C + q * nn, n, -1.0, 1.0, 0);
      }
      // Weyl widening of the leading bounds by every commutator term, ||M||_2 <= ||M||_F
      if (!(prob->e_max > prob->e_min)) {
        double* d_nrm = nullptr;
        if ((e = cudaMalloc(&d_nrm, 9 * sizeof(double))) != cudaSuccess) return fail(e, "cudaMalloc norms");
        cudaMemset(d_nrm, 0, 9 * sizeof(double));
        fq_launch_frobenius(K, nn, d_nrm, 0);
        for (int q = 0; q < 8; ++q) fq_launch_frobenius(C + q * nn, nn, d_nrm + 1 + q, 0);
        double nrm[9];
        e = cudaMemcpy(nrm, d_nrm, sizeof(nrm), cudaMemcpyDeviceToHost);
        cudaFree(d_nrm);
        if (e != cudaSuccess) return fail(e, "commutator norms");
        double wsum = 0.0;
        for (int q = 2; q < FQ_M6_TERMS; ++q) {
          double cmax = 0.0;
          for (int m = 0; m < M; ++m) cmax = std::max(cmax, fabs(p->coef6[(size_t)m * FQ_M6_TERMS + q]));
          wsum += cmax / p->h * sqrt(nrm[q - 2]);
        }
        if ((st = fq_finish_bounds(p, p->e_min - wsum, p->e_max + wsum)) != FQ_OK) return st;
      }
    }
  } else {
    if (p->order == 6) {  // the 6th-order basis as bands, computed on the host with the bounds
      if ((e = cudaMalloc(&p->d_cm, p->band6.size() * sizeof(double))) != cudaSuccess)
        return fail(e, "cudaMalloc basis bands");
      if ((e = cudaMemcpy(p->d_cm, p->band6.data(), p->band6.size() * sizeof(double), cudaMemcpyHostToDevice)) !=
          cudaSuccess)
        return fail(e, "upload basis bands");
    }
    std::vector<double> kl(std::max(1, n - 1), 0.0);
    for (int i = 0; i + 1 < n; ++i) kl[i] = prob->h0_off[i] * (prob->h1[i] - prob->h1[i + 1]);
    if ((e = cudaMalloc(&p->d_h0o, std::max(1, n - 1) * sizeof(double))) != cudaSuccess) return fail(e, "cudaMalloc H0 off");
    if (n > 1) {
      if ((e = cudaMemcpy(p->d_h0o, prob->h0_off, (n - 1) * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(e, "upload H0 off");
      if ((e = cudaMemcpy(p->d_k, kl.data(), (n - 1) * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(e, "upload K");
    }
  }
  if (p->path == PATH_DENSE_F64) {
    // small dense problems: one resident launch per chunk of steps instead of one per term
    const bool ok = fq_dense_resident_supported(n, p->L);
    const bool need = prob->kernel == FQ_KERNEL_RESIDENT || p->precision == FQ_DF32;
    if (need && !ok) {
      fq_set_error("dense resident kernel (and dense FQ_DF32) needs N <= 128 and L <= 128 (N = %d, L = %d)", n, p->L);
      return FQ_EUNSUPPORTED;
    }
    if (p->precision == FQ_DF32 && prob->kernel != FQ_KERNEL_AUTO && prob->kernel != FQ_KERNEL_RESIDENT) {
      fq_set_error("dense FQ_DF32 runs on the resident kernel only");
      return FQ_EUNSUPPORTED;
    }
    p->dense_resident = ok && (prob->kernel == FQ_KERNEL_AUTO || prob->kernel == FQ_KERNEL_RESIDENT);
  }
  *out = own.release();
  return FQ_OK;
}

}  // namespace

void fq_ktimer_start(const fq_plan* p, cudaStream_t s, const char* name) {
  fq_ktimer* t = p->ktimer;
  if (!t || !t->on || t->err != cudaSuccess) return;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return;
  try {
    while (t->ev.size() < t->used + 2) {
      cudaEvent_t e = nullptr;
      if ((t->err = cudaEventCreate(&e)) != cudaSuccess) return;
      t->ev.push_back(e);
    }
  } catch (...) {
    t->err = cudaErrorMemoryAllocation;
    return;
  }
  if ((t->err = cudaEventRecord(t->ev[t->used], s)) != cudaSuccess) return;
  t->name = name;
  t->open = true;
}

void fq_ktimer_stop(const fq_plan* p, cudaStream_t s) {
  fq_ktimer* t = p->ktimer;
  if (!t || !t->open) return;
  t->open = false;
  if ((t->err = cudaEventRecord(t->ev[t->used + 1], s)) == cudaSuccess) t->used += 2;
}

extern "C" {

fq_status floquet_plan_create(fq_plan** out, const fq_problem* prob) {
  if (!out) { fq_set_error("plan pointer is NULL"); return FQ_EINVAL; }
  *out = nullptr;
  return fq_guard("floquet_plan_create", [&] { return plan_create(out, prob); });
}

void floquet_plan_destroy(fq_plan* p) {
  if (!p) return;
  cudaDeviceSynchronize();
  free_plan(p);
}

fq_status floquet_plan_get_info(const fq_plan* p, fq_plan_info* info) {
  if (!p || !info) { fq_set_error("NULL argument"); return FQ_EINVAL; }
  info->n = p->n;
  info->steps = p->steps;
  info->L = p->L;
  info->precision = p->precision;
  info->format = p->format;
  info->drive_kind = p->drive_kind;
  info->h = p->h;
  info->e_min = p->e_min;
  info->e_max = p->e_max;
  info->beta = p->beta;
  info->delta_e = p->delta_e;
  info->R = p->R;
  return FQ_OK;
}

fq_status floquet_plan_inspect(const fq_problem* prob, fq_plan_info* info, double* coeffs, int32_t cap) {
  return fq_guard("floquet_plan_inspect", [&] {
    fq_plan p;
    fq_status st = fq_host_plan(prob, &p);
    if (st != FQ_OK) return st;
    st = floquet_plan_get_info(&p, info);
    if (coeffs)
      for (int l = 0; l <= p.L && l < cap; ++l) coeffs[l] = p.cheb[l];
    return st;
  });
}

size_t floquet_workspace_size(const fq_plan* p, int32_t ncols) {
  if (!p || ncols < 0) return 0;
  return layout(p, ncols, p->steps, nullptr, nullptr);
}

fq_status floquet_build_UT(fq_plan* p, void* d_U, void* d_ws, size_t ws_bytes, void* stream) {
  if (!p || !d_U) { fq_set_error("NULL plan or output"); return FQ_EINVAL; }
  return propagate_impl(p, nullptr, (double*)d_U, p->n, 0, p->steps, 1, 1, d_ws, ws_bytes, (cudaStream_t)stream);
}

fq_status floquet_build_UT_report(fq_plan* p, void* d_U, void* d_ws, size_t ws_bytes, void* stream,
                                  int32_t defect_columns, fq_report* rep) {
  if (!p || !d_U || !rep) { fq_set_error("NULL plan, output or report"); return FQ_EINVAL; }
  const int n = p->n;
  if (defect_columns < 1 || defect_columns > n) {
    fq_set_error("floquet_build_UT_report: defect_columns must be in [1, %d] (got %d)", n, defect_columns);
    return FQ_EINVAL;
  }
  const size_t dws = floquet_defect_workspace_size(n), need = dws + align_up(4 * (size_t)defect_columns);
  if (!d_ws || ws_bytes < need) {
    fq_set_error("floquet_build_UT_report: workspace must hold %zu bytes for the defect", need);
    return FQ_EINVAL;
  }
  return fq_guard("floquet_build_UT_report", [&]() -> fq_status {
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce == cudaSuccess) ce = cudaEventRecord(e0, s);
    fq_status st = ce == cudaSuccess ? floquet_build_UT(p, d_U, d_ws, ws_bytes, stream) : fq_cuda_fail(ce, "events");
    if (st == FQ_OK && (ce = cudaEventRecord(e1, s)) != cudaSuccess) st = fq_cuda_fail(ce, "event record");
    // the workspace is free again: the defect's partial sums, then the column list
    std::vector<int32_t> cols(defect_columns);
    for (int q = 0; q < defect_columns; ++q) cols[q] = (int32_t)(((int64_t)q * n) / defect_columns);
    int32_t* d_cols = (int32_t*)((char*)d_ws + dws);
    if (st == FQ_OK && (ce = cudaMemcpyAsync(d_cols, cols.data(), 4 * cols.size(), cudaMemcpyHostToDevice, s)) !=
                           cudaSuccess)
      st = fq_cuda_fail(ce, "defect columns");
    double mx = 0.0, fro = 0.0;
    if (st == FQ_OK) st = floquet_unitarity_defect(d_U, n, d_cols, defect_columns, d_ws, dws, stream, &mx, &fro);
    float ms = 0.f;
    if (st == FQ_OK && (ce = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) st = fq_cuda_fail(ce, "event time");
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st != FQ_OK) return st;
    rep->L = p->L;
    rep->defect_columns = defect_columns;
    rep->R = p->R;
    rep->e_min = p->e_min;
    rep->e_max = p->e_max;
    rep->beta = p->beta;
    rep->delta_e = p->delta_e;
    rep->defect_max = mx;
    rep->defect_fro = fro;
    rep->build_ms = ms;
    return floquet_check_status(p, stream);
  });
}

fq_status floquet_kernel_timing(fq_plan* p, int32_t enable) {
  if (!p) { fq_set_error("NULL plan"); return FQ_EINVAL; }
  return fq_guard("floquet_kernel_timing", [&]() -> fq_status {
    if (!p->ktimer) p->ktimer = new fq_ktimer();
    fq_ktimer* t = p->ktimer;
    t->on = enable != 0;
    t->open = false;
    t->used = 0;
    t->err = cudaSuccess;
    t->name = "";
    return FQ_OK;
  });
}

fq_status floquet_kernel_time(fq_plan* p, int32_t* launches, double* total_ms, char* name, int32_t name_len) {
  if (!p || !launches || !total_ms) { fq_set_error("NULL plan or output"); return FQ_EINVAL; }
  *launches = 0;
  *total_ms = 0.0;
  if (name && name_len > 0) name[0] = '\0';
  fq_ktimer* t = p->ktimer;
  if (!t) return FQ_OK;
  const size_t used = t->used;
  const cudaError_t failed = t->err;
  t->used = 0;
  t->err = cudaSuccess;
  if (failed != cudaSuccess) return fq_cuda_fail(failed, "kernel timing events");
  double sum = 0.0;
  if (used > 0) {
    cudaError_t e = cudaEventSynchronize(t->ev[used - 1]);
    for (size_t k = 0; k < used && e == cudaSuccess; k += 2) {
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, t->ev[k], t->ev[k + 1]);
      sum += ms;
    }
    if (e != cudaSuccess) return fq_cuda_fail(e, "kernel timing");
  }
  *launches = (int32_t)(used / 2);
  *total_ms = sum;
  if (name && name_len > 0) snprintf(name, (size_t)name_len, "%s", used ? t->name : "");
  return FQ_OK;
}

fq_status floquet_propagate(fq_plan* p, const void* d_X0, void* d_X, int32_t ncols, int32_t m_begin, int32_t m_end,
                            void* d_ws, size_t ws_bytes, void* stream) {
  if (!p || !d_X0 || !d_X) { fq_set_error("NULL plan or state pointer"); return FQ_EINVAL; }
  if (ncols < 0 || m_begin < 0 || m_end > p->steps || m_begin > m_end) {
    fq_set_error("bad range: ncols %d, steps [%d, %d) of %d", ncols, m_begin, m_end, p->steps);
    return FQ_EINVAL;
  }
  if (m_begin == m_end) {
    if (d_X != d_X0)
      return cuda_ok(cudaMemcpyAsync(d_X, d_X0, (size_t)ncols * p->n * 16, cudaMemcpyDeviceToDevice,
                                     (cudaStream_t)stream), "copy");
    return FQ_OK;
  }
  return propagate_impl(p, (const double*)d_X0, (double*)d_X, ncols, m_begin, m_end, 0, 0, d_ws, ws_bytes,
                        (cudaStream_t)stream);
}

size_t floquet_columns_workspace_size(const fq_plan* p, int32_t ncols) {
  if (!p || ncols < 1) return 0;
  return align_up((size_t)ncols * p->n * 16) + layout(p, ncols, p->steps, nullptr, nullptr);
}

fq_status floquet_build_UT_columns(fq_plan* p, int32_t j0, int32_t ncols, void* d_X, void* d_ws, size_t ws_bytes,
                                   void* stream) {
  if (!p || !d_X) { fq_set_error("NULL plan or output"); return FQ_EINVAL; }
  if (ncols < 1 || j0 < 0 || (int64_t)j0 + ncols > p->n) {
    fq_set_error("floquet_build_UT_columns: columns [%d, %lld) outside [0, %d)", j0, (long long)j0 + ncols, p->n);
    return FQ_EINVAL;
  }
  const size_t head = align_up((size_t)ncols * p->n * 16);
  if (!d_ws || ws_bytes < head || ((uintptr_t)d_ws & (kAlign - 1))) {
    fq_set_error("floquet_build_UT_columns: workspace must be >= %zu bytes, 256-byte aligned",
                 floquet_columns_workspace_size(p, ncols));
    return FQ_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  double* x0 = (double*)d_ws;
  fq_launch_basis_rows(x0, ncols, p->n, j0, s);
  return propagate_impl(p, x0, (double*)d_X, ncols, 0, p->steps, 0, 0, (char*)d_ws + head, ws_bytes - head, s);
}

size_t floquet_defect_workspace_size(int32_t n) {
  if (n < 1) return 0;
  return align_up(2 * sizeof(double) * (size_t)((n + 15) / 16) * ((n + 255) / 256));
}

fq_status floquet_unitarity_defect(const void* d_U, int32_t n, const int32_t* d_cols, int32_t k, void* d_ws,
                                   size_t ws_bytes, void* stream, double* max_abs, double* fro) {
  if (!d_U || n < 1 || !max_abs || !fro) { fq_set_error("bad defect arguments"); return FQ_EINVAL; }
  const int rows = d_cols ? k : n;
  if (rows < 1 || rows > n) { fq_set_error("defect: k must be in [1, n]"); return FQ_EINVAL; }
  const int nb = (n + 255) / 256;
  const int chunks = (rows + 15) / 16;
  const size_t need = align_up(2 * sizeof(double) * (size_t)chunks * nb);
  if (!d_ws || ws_bytes < need) { fq_set_error("defect workspace too small (%zu < %zu)", ws_bytes, need); return FQ_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  fq_launch_defect((const double*)d_U, n, d_cols, rows, (double*)d_ws, s);
  std::vector<double> h(2 * (size_t)chunks * nb, 0.0);  // at most 2 * 16 * N / 256 doubles: N ~ 10^4 is 2.5 KB
  cudaError_t e = cudaMemcpyAsync(h.data(), d_ws, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fq_cuda_fail(e, "defect");
  double mx = 0.0, ss = 0.0;
  for (size_t q = 0; q < h.size(); q += 2) {
    mx = std::max(mx, h[q]);
    ss += h[q + 1];
  }
  *max_abs = mx;
  *fro = sqrt(ss / rows);  // Frobenius norm of the k rows of U^+U - 1, over sqrt(k)
  return FQ_OK;
}

fq_status floquet_selftest_wait(fq_plan* p, int64_t cycles, void* stream) {
  if (!p || cycles < 1 || cycles > (1ll << 31)) {
    fq_set_error("floquet_selftest_wait: needs a plan and 1 <= cycles <= 2^31");
    return FQ_EINVAL;
  }
  fq_launch_wait_probe(p->d_status, (long long)cycles, (cudaStream_t)stream);
  return cuda_ok(cudaGetLastError(), "wait probe");
}

fq_status floquet_probe_fp32(int32_t packed, int32_t iters, float* d_out, int64_t out_len, void* stream,
                             double* flops) {
  const int64_t blocks = std::min<int64_t>(4LL * fq_sm_count(), out_len / 256);
  if (!d_out || !flops || iters < 1 || blocks < 1) {
    fq_set_error("floquet_probe_fp32: needs iters >= 1, flops and a device buffer of >= 256 floats");
    return FQ_EINVAL;
  }
  *flops = fq_launch_fp32_probe(packed != 0, iters, d_out, (int)blocks, (cudaStream_t)stream);
  return cuda_ok(cudaGetLastError(), "FP32 probe");
}

fq_status floquet_check_status(fq_plan* p, void* stream) {
  if (!p) { fq_set_error("NULL plan"); return FQ_EINVAL; }
  unsigned int v = 0;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(&v, p->d_status, sizeof(v), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fq_cuda_fail(e, "status read");
  if (v) {
    cudaMemsetAsync(p->d_status, 0, sizeof(unsigned int), s);
    cudaStreamSynchronize(s);
    if (v & FQ_BIT_TIMEOUT) { fq_set_error("a bounded device wait timed out"); return FQ_ETIMEOUT; }
    fq_set_error("device check: an entry exceeded the unitarity bound or was NaN (spectral bounds too tight?)");
    return FQ_EBOUND;
  }
  return FQ_OK;
}

}  // extern "C"
