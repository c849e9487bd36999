// Quasienergies and Floquet states from U_T on the host (Eq. 5: U_T phi_mu = e^{-i eps_mu T} phi_mu),
// outside the timed propagation.  No LAPACK is linked, so the complex Schur form is computed here
// by the textbook route (Golub and Van Loan, "Matrix Computations", §7.4-7.5): Householder
// reduction to upper Hessenberg form, then single-shift QR sweeps with Givens rotations, a
// Wilkinson shift from the trailing 2 x 2 block, an exceptional shift every 10 sweeps without
// deflation, and deflation at |h_{k+1,k}| <= eps (|h_kk| + |h_{k+1,k+1}|).  U_T is unitary,
// hence normal, so its Schur form is diagonal to rounding and the accumulated Schur vectors are
// the Floquet states.  O(N^3), built with -fcx-limited-range (U_T is unitary, so no complex
// product comes near overflow).  The row-independent updates (Householder, the R Q half of each
// sweep, the Schur vectors) run on up to 16 threads; the Q R rotations of a sweep form one
// dependency chain and stay on the calling thread.  On 8 x86 cores: about 0.6 s at N = 512 and
// 3.5 s at N = 1000 for the quasienergies alone, 1 s and 4.7 s with the states.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <complex>
#include <condition_variable>
#include <functional>
#include <memory>
#include <mutex>
#include <numeric>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

using cd = std::complex<double>;

// Wilkinson shift: the eigenvalue of [[a, b], [c, d]] closer to d.
cd wilkinson(cd a, cd b, cd c, cd d) {
  const cd tr = a + d, det = a * d - b * c;
  const cd disc = std::sqrt(tr * tr - 4.0 * det);
  const cd l1 = 0.5 * (tr + disc), l2 = 0.5 * (tr - disc);
  return std::abs(l1 - d) < std::abs(l2 - d) ? l1 : l2;
}

// Givens rotation [c s; -conj(s) c] (c real) with [c s; -conj(s) c] [x; y] = [r; 0].
void givens(cd x, cd y, double& c, cd& s) {
  const double ax = std::abs(x), ay = std::abs(y);
  if (ay == 0.0) {
    c = 1.0;
    s = 0.0;
    return;
  }
  if (ax == 0.0) {
    c = 0.0;
    s = std::conj(y) / ay;
    return;
  }
  const double nrm = std::hypot(ax, ay);
  c = ax / nrm;
  s = (x / ax) * std::conj(y) / nrm;
}

// Worker threads that share the row-independent updates of one step: run(count, f) calls
// f(lo, hi) on contiguous slices of [0, count), one slice per thread (the caller takes the
// first), and returns when every slice is done.  Each row or column is handled by one thread in
// the serial order, so the results do not depend on the number of threads.
class RowPool {
 public:
  explicit RowPool(int nthreads) : nt_(std::max(1, nthreads)) {
    for (int t = 1; t < nt_; ++t) workers_.emplace_back([this, t] { loop(t); });
  }
  ~RowPool() {
    {
      std::lock_guard<std::mutex> g(mu_);
      stop_ = true;
      ++gen_;
    }
    cv_.notify_all();
    for (auto& w : workers_) w.join();
  }
  void run(int count, const std::function<void(int, int)>& f) {
    {
      std::lock_guard<std::mutex> g(mu_);
      task_ = &f;
      count_ = count;
      pending_ = nt_ - 1;
      ++gen_;
    }
    cv_.notify_all();
    slice(0, f, count);
    std::unique_lock<std::mutex> g(mu_);
    done_.wait(g, [this] { return pending_ == 0; });
    task_ = nullptr;
  }

 private:
  void slice(int t, const std::function<void(int, int)>& f, int count) const {
    const int lo = (int)((long long)count * t / nt_), hi = (int)((long long)count * (t + 1) / nt_);
    if (lo < hi) f(lo, hi);
  }
  void loop(int t) {
    int seen = 0;
    for (;;) {
      const std::function<void(int, int)>* f;
      int count;
      {
        std::unique_lock<std::mutex> g(mu_);
        cv_.wait(g, [&] { return gen_ != seen; });
        seen = gen_;
        if (stop_) return;
        f = task_;
        count = count_;
      }
      slice(t, *f, count);
      std::lock_guard<std::mutex> g(mu_);
      if (--pending_ == 0) done_.notify_one();
    }
  }
  const int nt_;
  std::vector<std::thread> workers_;
  std::mutex mu_;
  std::condition_variable cv_, done_;
  const std::function<void(int, int)>* task_ = nullptr;
  int count_ = 0, pending_ = 0, gen_ = 0;
  bool stop_ = false;
};

struct Schur {
  int n;
  RowPool* pool = nullptr;  // NULL: every update on the calling thread
  std::vector<cd> H;  // row-major
  std::vector<cd> Q;  // row-major, accumulated when `vectors`
  bool vectors;
  cd& h(int i, int j) { return H[(size_t)i * n + j]; }
  cd& q(int i, int j) { return Q[(size_t)i * n + j]; }

  // f(lo, hi) over [0, count): on the pool when the update touches enough elements to pay for
  // the hand-off (a few microseconds), else here
  void par(int count, double elements, const std::function<void(int, int)>& f) {
    if (pool && count > 1 && elements >= 65536.0) pool->run(count, f);
    else if (count > 0) f(0, count);
  }

  // rows i0..i1 of M (row-major, n columns) times the rotations k = lo..hi-1 on columns k, k+1,
  // in order; row i only from rotation max(lo, kmin(i)) on.  Rows do not interact, so each
  // row takes its rotations in turn: the same arithmetic as rotation by rotation, along the row.
  template <class KMin>
  void rotate_columns(cd* M, int i0, int i1, int lo, int hi, const double* cs, const cd* sn, KMin kmin) {
    for (int i = i0; i <= i1; ++i) {
      cd* r = M + (size_t)i * n;
      for (int k = std::max(lo, kmin(i)); k < hi; ++k) {
        const cd a = r[k], b = r[k + 1];
        r[k] = cs[k] * a + std::conj(sn[k]) * b;
        r[k + 1] = -sn[k] * a + cs[k] * b;
      }
    }
  }

  // Householder reduction: H <- P^H H P, Q <- Q P
  void hessenberg() {
    std::vector<cd> v(n), w(n);
    for (int k = 0; k + 2 < n; ++k) {
      double norm2 = 0.0;
      for (int i = k + 1; i < n; ++i) norm2 += std::norm(h(i, k));
      const double xnorm = std::sqrt(norm2);
      if (xnorm == 0.0) continue;
      const cd x0 = h(k + 1, k);
      const cd phase = std::abs(x0) > 0 ? x0 / std::abs(x0) : cd(1.0, 0.0);
      const cd alpha = -phase * xnorm;
      for (int i = 0; i < n; ++i) v[i] = 0.0;
      v[k + 1] = x0 - alpha;
      for (int i = k + 2; i < n; ++i) v[i] = h(i, k);
      double vv = 0.0;
      for (int i = k + 1; i < n; ++i) vv += std::norm(v[i]);
      if (vv == 0.0) continue;
      const double beta = 2.0 / vv;  // P = I - beta v v^H
      // left: H <- P H on rows k+1.., columns k..; w_j = sum_i conj(v_i) h_ij by column slices
      // (each w_j summed over i in order), then the rank-one update by rows
      const int m = n - k;
      const double area = (double)m * m;
      par(m, area, [&](int j0, int j1) {
        for (int j = k + j0; j < k + j1; ++j) w[j] = 0.0;
        for (int i = k + 1; i < n; ++i) {
          const cd vi = std::conj(v[i]);
          const cd* r = &h(i, 0);
          for (int j = k + j0; j < k + j1; ++j) w[j] += vi * r[j];
        }
      });
      par(m - 1, area, [&](int i0, int i1) {
        for (int i = k + 1 + i0; i < k + 1 + i1; ++i) {
          const cd f = beta * v[i];
          cd* r = &h(i, 0);
          for (int j = k; j < n; ++j) r[j] -= f * w[j];
        }
      });
      // right: H <- H P on all rows, columns k+1..; Q <- Q P likewise
      const auto right = [&](cd* M) {
        par(n, (double)n * m, [&, M](int i0, int i1) {
          for (int i = i0; i < i1; ++i) {
            cd* r = M + (size_t)i * n;
            cd s = 0.0;
            for (int j = k + 1; j < n; ++j) s += r[j] * v[j];
            s *= beta;
            for (int j = k + 1; j < n; ++j) r[j] -= s * std::conj(v[j]);
          }
        });
      };
      right(H.data());
      if (vectors) right(Q.data());
      for (int i = k + 2; i < n; ++i) h(i, k) = 0.0;
    }
  }

  // shifted QR sweeps to upper triangular form; false if it does not converge
  bool qr() {
    const double eps = 2.220446049250313e-16;
    int hi = n - 1, iter = 0, total = 0;
    std::vector<double> cs(n);
    std::vector<cd> sn(n);
    while (hi > 0) {
      int lo = hi;
      while (lo > 0) {
        const double tol = eps * (std::abs(h(lo - 1, lo - 1)) + std::abs(h(lo, lo)));
        if (std::abs(h(lo, lo - 1)) <= std::max(tol, 1e-300)) {
          h(lo, lo - 1) = 0.0;
          break;
        }
        --lo;
      }
      if (lo == hi) {
        --hi;
        iter = 0;
        continue;
      }
      if (++total > 60 * n) return false;
      ++iter;
      cd mu = wilkinson(h(hi - 1, hi - 1), h(hi - 1, hi), h(hi, hi - 1), h(hi, hi));
      if (iter % 10 == 0) mu = h(hi, hi) + std::abs(h(hi, hi - 1));  // exceptional shift
      for (int k = lo; k <= hi; ++k) h(k, k) -= mu;
      // H - mu I = Q R: rotations on rows k, k+1 over columns k..hi.  Only the diagonal of the
      // Schur form is read and the rotations depend on the active block alone, so H is updated
      // inside rows/columns lo..hi only, with or without the Schur vectors.
      for (int k = lo; k < hi; ++k) {
        givens(h(k, k), h(k + 1, k), cs[k], sn[k]);
        const double c = cs[k];
        const cd s = sn[k];
        for (int j = k; j <= hi; ++j) {
          const cd a = h(k, j), b = h(k + 1, j);
          h(k, j) = c * a + s * b;
          h(k + 1, j) = -std::conj(s) * a + c * b;
        }
      }
      // R Q: the transposed rotations on columns k, k+1 over rows lo..k+1 (row i from k = i - 1),
      // and on the same columns of Q over all rows
      const int m = hi - lo + 1;
      par(m, 0.5 * m * m, [&](int i0, int i1) {
        rotate_columns(H.data(), lo + i0, lo + i1 - 1, lo, hi, cs.data(), sn.data(), [](int i) { return i - 1; });
      });
      if (vectors)
        par(n, (double)n * m, [&](int i0, int i1) {
          rotate_columns(Q.data(), i0, i1 - 1, lo, hi, cs.data(), sn.data(), [](int) { return 0; });
        });
      for (int k = lo; k <= hi; ++k) h(k, k) += mu;
    }
    return true;
  }
};

}  // namespace

static fq_status floquet_quasienergies_body(const void* U, int32_t n, double period, double* eps_out,
                                            void* states_out) {
  if (!U || !eps_out || n < 1 || !(period > 0)) {
    fq_set_error("floquet_quasienergies: needs U, eps_out, n >= 1 and period > 0");
    return FQ_EINVAL;
  }
  Schur s;
  s.n = n;
  // threads for the row updates: up to 16, and none below N = 128 (one step's update is then
  // too small to share)
  const int nt = n >= 128 ? (int)std::min<unsigned>(16, std::max(1u, std::thread::hardware_concurrency())) : 1;
  std::unique_ptr<RowPool> pool(nt > 1 ? new RowPool(nt) : nullptr);
  s.pool = pool.get();
  s.vectors = states_out != nullptr;
  s.H.assign((const cd*)U, (const cd*)U + (size_t)n * n);
  if (s.vectors) {
    s.Q.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) s.q(i, i) = 1.0;
  }
  s.hessenberg();
  if (!s.qr()) {
    fq_set_error("floquet_quasienergies: the QR iteration did not converge");
    return FQ_EINVAL;
  }
  // theta = -arg(lambda) folded into [-pi, pi), eps = theta / T, ascending
  std::vector<double> eps(n);
  for (int k = 0; k < n; ++k) {
    double th = -std::arg(s.h(k, k));
    if (th >= M_PI) th -= 2.0 * M_PI;
    eps[k] = th / period;
  }
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return eps[a] < eps[b]; });
  for (int k = 0; k < n; ++k) eps_out[k] = eps[order[k]];
  if (s.vectors) {
    cd* out = (cd*)states_out;  // row mu = Floquet state of eps_out[mu] (a Schur vector)
    for (int mu = 0; mu < n; ++mu)
      for (int i = 0; i < n; ++i) out[(size_t)mu * n + i] = s.q(i, order[mu]);
  }
  return FQ_OK;
}

extern "C" fq_status floquet_quasienergies(const void* U, int32_t n, double period, double* eps_out,
                                           void* states_out) {
  return fq_guard("floquet_quasienergies", [&] {
    return floquet_quasienergies_body(U, n, period, eps_out, states_out);
  });
}
