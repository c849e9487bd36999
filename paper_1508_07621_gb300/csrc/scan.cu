// Batched scan: the U_T builds of many independent split-precision dense plans as ONE persistent
// tcgen05 launch (stages a2, a3, a5, a6 and a8 of every instance, Eqs. 10-14).
//
// Work units, in one global order that every dependency respects (a unit waits only on units
// that come before it):
//   prologue  B(i, 0, b)     instance i, block b of 16 rows: the identity's left-operand slices and
//                            FP32 masters, and the S and A slices of Omega~_0 (Eqs. 11 and 14);
//   step m    T(i, m, p, t)  term p of step m of instance i (Eq. 10) on output tile t (128 states x
//                            BN rows of Omega~), term p of every instance before term p + 1;
//             B(i, m + 1, b) the slices of Omega~_{m+1}, in shares after the instance's terms
//                            1 .. L - 1;
//   end       W(i, b)        16 states of U_T: FP32 masters to complex128, transposed.
// CTAs take units from a device counter, so cheap and costly instances balance.  Units are taken in
// increasing order and each waits only on earlier ones, so the scan always advances, whether or not
// every CTA is resident.  In each CTA a TMA producer thread takes the units and hands them through
// a ring of SCAN_RING slots in shared memory to the MMA thread, four epilogue warps and four
// builder warps.  The term units run as in k_split_chain (two accumulator buffers in tensor memory,
// the epilogue of one tile overlapping the MMAs of the next); the builder warps do the B and W
// units beside them, so that their memory latency stays off the tensor cores' path.
// Dependencies (monotonic counters in global memory, bounded acquire spins):
//   T(i, m, p, tile of state block tj): every B(i, m, *) done (a counter per buffer parity: Omega~_m
//     lives in buffer m & 1), and term p - 1 of step m (term L - 1 of step m - 1 when p = 0) done on
//     state block tj (its four epilogue warps per tile, counted per (i, p, tj) across the steps);
//   B(i, m, *), m >= 2: step m - 2 done on every state block (its buffer has been read);
//   W(i, b): step M - 1 done on the state block of its 16 states.
// The arithmetic of every unit is that of the one-instance path (dense_split.cu) with the same tile
// shape, so each instance's U_T equals its own floquet_build_UT bit for bit.
#include <algorithm>
#include <climits>
#include <numeric>
#include <vector>

#include "split_core.cuh"

namespace {

constexpr int SCAN_MAXL = 32;    // Chebyshev terms per step an instance may have
constexpr int SCAN_RING = 8;     // units handed from the producer to the MMA thread and the warps
constexpr int SCAN_THREADS = 320;  // producer, MMA, four epilogue warps, four builder warps
constexpr int BLOCK_ROWS = 16;   // rows of a B or W unit
constexpr int SCAN_TAIL = 512;   // barriers, tensor-memory slot, abort flag and ring after the stages

enum ScanUnitType { SU_TERM = 0, SU_OMEGA = 1, SU_STORE = 2, SU_END = 3 };

struct ScanInst {  // 128-byte aligned through its tensor maps
  CUtensorMap a[2][3];     // left-operand slices [np][2 np], buffers 0 and 1
  CUtensorMap os[2][3];    // S slices of Omega~_m [np][np], buffer m & 1
  CUtensorMap oa[2][3];    // A slices
  const double* h0;        // N x N operators and [H0, H1]
  const double* h1;
  const double* k;
  const double* scal;      // per-step scalars: sa [M] | sb [M] | sc [M]
  __nv_bfloat16* os_buf[2];
  __nv_bfloat16* oa_buf[2];
  __nv_bfloat16* abuf[2];
  float* m[3][2];          // FP32 masters (re, im), [n][ldm]
  double2* u;              // output U_T, N x N complex128
  unsigned int* status;
  unsigned int* termcnt;   // [L][tiles_j]
  unsigned int* omegacnt;  // [2]: finished B-unit epilogue warps writing buffer 0 / 1
  double cheb[SCAN_MAXL + 1];
  double sbeta, ph_re, ph_im;
  size_t bstride, astride;
  int n, ldm, np, kp, L, tiles_i, tiles_j, nk, nblk, steps;
};

// A run of consecutive units of one kind and instance; `begin` counts from the start of its table
// (prologue, one step, or end).  p: the term (SU_TERM) or the first 16-row block (SU_OMEGA).
struct ScanSeg {
  int begin, type, inst, p;
};

struct ScanArgs {
  const ScanInst* inst;
  const ScanSeg* seg;      // prologue [0, npro), one step [npro, npro + nstep), end [.., + nend)
  int npro, nstep, nend;
  int upro, ustep, uend, steps, count, total;
  unsigned int* next;      // unit counter
  int* abort;              // set by the first CTA that gives up
};

struct ScanUnit {
  int type, inst, m, p, t;
};

__device__ __forceinline__ ScanUnit scan_decode(const ScanArgs& a, int u) {
  ScanUnit d{SU_END, 0, 0, 0, 0};
  if (u < 0 || u >= a.total) return d;
  int r = u, lo = 0, hi = a.npro, m = 0;
  if (u >= a.upro) {
    r = u - a.upro;
    m = r / a.ustep;
    if (m < a.steps) {
      r -= m * a.ustep;
      lo = a.npro;
      hi = a.npro + a.nstep;
    } else {
      r -= a.steps * a.ustep;
      lo = a.npro + a.nstep;
      hi = lo + a.nend;
    }
  }
  while (hi - lo > 1) {  // last segment that starts at or before r
    const int mid = (lo + hi) >> 1;
    if (a.seg[mid].begin <= r) lo = mid;
    else hi = mid;
  }
  const ScanSeg s = a.seg[lo];
  d.type = s.type;
  d.inst = s.inst;
  d.p = s.type == SU_TERM ? s.p : 0;
  d.t = r - s.begin + (s.type == SU_OMEGA ? s.p : 0);  // an Omega~ run starts at block s.p
  d.m = u < a.upro ? 0 : (s.type == SU_OMEGA ? m + 1 : m);
  return d;
}

// bounded wait until *p >= target (acquire); false if it gave up or the scan was aborted
__device__ __forceinline__ bool scan_wait(const unsigned int* p, unsigned int target, const int* gabort) {
  const long long t0 = clock64();
  while (ld_acquire_u32(p) < target) {
    if (*(const volatile int*)gabort || clock64() - t0 > kWaitCycles) return false;
    __nanosleep(64);
  }
  return true;
}

// bounded mbarrier wait that also gives up once `flag` is set
__device__ __forceinline__ bool mbar_wait_or(uint32_t bar, uint32_t parity, const int* flag) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (*(const volatile int*)flag || clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}

// Epilogue of term p of step m: the three FP32 master buffers rotate as in dense_split.cu (psi_0
// in buffer A = (m (L mod 2)) mod 3, psi_1, psi_3, ... in B = A + 1, psi_2, psi_4, ... in A,
// the Bessel sum in C = A + 2), and the left-operand buffers alternate term by term.
__device__ __forceinline__ void scan_epi(const ScanInst& I, int m, int p, SplitEpi& e) {
  const int rot = m * (I.L & 1);
  const int A = rot % 3, B = (rot + 1) % 3, C = (rot + 2) % 3;
  const int av = (rot & 1) ^ (p & 1);
  int cur = A, prv = A, out = B;
  if (p > 0) {
    cur = (p & 1) ? B : A;
    prv = (p & 1) ? A : B;
    out = prv;
  }
  e = SplitEpi{};
  e.n = I.n;
  e.nc = I.n;
  e.ldm = I.ldm;
  e.np = I.np;
  e.kp = I.kp;
  e.cur_re = I.m[cur][0];
  e.cur_im = I.m[cur][1];
  e.prev_re = I.m[prv][0];
  e.prev_im = I.m[prv][1];
  e.acc_re = I.m[C][0];
  e.acc_im = I.m[C][1];
  e.out_re = I.m[out][0];
  e.out_im = I.m[out][1];
  e.slice_out = I.abuf[av ^ 1];
  e.slice_stride = I.astride;
  e.t.first = p == 0;
  e.t.last = p == I.L - 1;
  e.t.coef0 = I.cheb[0];
  e.t.coef = I.cheb[p + 1];
  e.t.ph_re = I.ph_re;
  e.t.ph_im = I.ph_im;
  e.t.bound2 = 1.0 + 2e-3;
  e.t.status = I.status;
}

// B unit: rows [r0, r0 + 16) of Omega~_m's S and A slices (buffer m & 1), as k_split_omega; at
// m = 0 also the same rows of the identity block's left operand (buffer 0) and masters (buffer
// 0), as k_split_init, and zeros in left-operand buffer 1.
template <int NS>
__device__ void scan_omega_rows(const ScanInst& I, int m, int r0, int tid) {
  const int n = I.n, np = I.np, M = I.steps;
  const float sa = (float)I.scal[m], sb = (float)I.scal[M + m], sc = (float)I.scal[2 * M + m];
  const float sbeta = (float)I.sbeta;
  __nv_bfloat16* os = I.os_buf[m & 1];
  __nv_bfloat16* oa = I.oa_buf[m & 1];
  // 8 entries a thread per pass, their 24 loads issued before any use (the unit is latency-bound
  // otherwise); BLOCK_ROWS * np is a multiple of 128 * 8 since np is a multiple of 128
  constexpr int U = 8;
  int i = r0 + tid / np, c = tid % np;
  for (int q0 = 0; q0 < BLOCK_ROWS * np; q0 += 4 * 32 * U) {
    double x0[U], x1[U], xk[U];
    int ii[U], cc[U];
#pragma unroll
    for (int s = 0; s < U; ++s) {
      ii[s] = i;
      cc[s] = c;
      const bool in = i < n && c < n;
      const size_t o = (size_t)i * n + c;
      x0[s] = in ? __ldg(I.h0 + o) : 0.0;
      x1[s] = in ? __ldg(I.h1 + o) : 0.0;
      xk[s] = in ? __ldg(I.k + o) : 0.0;
      c += 4 * 32;  // the next entry of this thread: 128 further on, at most one row on (np >= 128)
      if (c >= np) {
        c -= np;
        ++i;
      }
    }
#pragma unroll
    for (int s = 0; s < U; ++s) {
      float S = 0.f, A = 0.f;
      if (ii[s] < n && cc[s] < n) omega_entry(x0[s], x1[s], xk[s], ii[s] == cc[s], sa, sb, sc, sbeta, S, A);
      __nv_bfloat16 s1[NS], s2[NS];
      split_f32<NS>(S, s1);
      split_f32<NS>(A, s2);
      const size_t e = (size_t)ii[s] * np + cc[s];
#pragma unroll
      for (int t = 0; t < NS; ++t) {
        os[t * I.bstride + e] = s1[t];
        oa[t * I.bstride + e] = s2[t];
      }
    }
  }
  if (m != 0) return;
  const int kp = I.kp;
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
  for (int q = tid; q < BLOCK_ROWS * kp; q += 4 * 32) {
    const int j = r0 + q / kp, c = q % kp;
    const bool im_half = c >= np;
    const int i = im_half ? c - np : c;
    float v = 0.f;
    if (j < n && i < n) {
      v = (!im_half && i == j) ? 1.f : 0.f;
      if (im_half) I.m[0][1][(size_t)j * I.ldm + i] = v;
      else I.m[0][0][(size_t)j * I.ldm + i] = v;
    }
    __nv_bfloat16 s[NS];
    split_f32<NS>(v, s);
    const size_t e = (size_t)j * kp + c;
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      I.abuf[0][t * I.astride + e] = s[t];
      I.abuf[1][t * I.astride + e] = zero;
    }
  }
}

// W unit: U[i][j] = X_j[i] for the states j in [j0, j0 + 16), X = the masters after step M - 1.
__device__ void scan_store_rows(const ScanInst& I, int j0, int tid) {
  const int n = I.n, xb = (I.steps * (I.L & 1)) % 3;
  const float* xr = I.m[xb][0];
  const float* xi = I.m[xb][1];
  const int cnt = min(BLOCK_ROWS, n - j0);
  for (int i = tid; i < n; i += 4 * 32) {
    float vr[BLOCK_ROWS], vi[BLOCK_ROWS];
#pragma unroll
    for (int r = 0; r < BLOCK_ROWS; ++r) {
      const size_t s = (size_t)(j0 + r) * I.ldm + i;
      vr[r] = r < cnt ? xr[s] : 0.f;
      vi[r] = r < cnt ? xi[s] : 0.f;
    }
#pragma unroll
    for (int r = 0; r < BLOCK_ROWS; ++r)
      if (r < cnt) I.u[(size_t)i * n + j0 + r] = make_double2((double)vr[r], (double)vi[r]);
  }
}

template <int NS, int BN, int BKE>
struct ScanCfg {
  using Split = SplitCfg<NS, BN, BKE, true>;
  static constexpr size_t SMEM = (size_t)Split::STAGES * Split::STAGE_BYTES + 1024 + SCAN_TAIL;
};

template <int NS, int BN, int BKE>
__global__ void __launch_bounds__(SCAN_THREADS, 1) k_split_scan(const __grid_constant__ ScanArgs a) {
  using Cfg = SplitCfg<NS, BN, BKE, true>;
  constexpr int STAGES = Cfg::STAGES;
  constexpr int R = SCAN_RING;
  constexpr uint32_t BUF_COLS = 2 * BN;
  constexpr uint32_t TMEM_COLS = 2 * BUF_COLS;
  static_assert((2 * STAGES + 5 + 2 * R) * 8 + 8 + R * 5 * 4 <= SCAN_TAIL, "shared tail");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = smem_raw + (base - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + STAGES * Cfg::STAGE_BYTES);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES);
  const uint32_t tfull0 = smem_u32(bars + 2 * STAGES), tempty0 = smem_u32(bars + 2 * STAGES + 2);
  const uint32_t done = smem_u32(bars + 2 * STAGES + 4);
  const uint32_t ufull0 = smem_u32(bars + 2 * STAGES + 5), uempty0 = smem_u32(bars + 2 * STAGES + 5 + R);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 5 + 2 * R);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  volatile int* ring = reinterpret_cast<volatile int*>(tmem_slot + 2);  // [R][5]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull0 + 8 * b, 1);
      mbar_init(tempty0 + 8 * b, 4);
    }
    mbar_init(done, 1);
    for (int s = 0; s < R; ++s) {
      mbar_init(ufull0 + 8 * s, 1);
      mbar_init(uempty0 + 8 * s, 9);  // the MMA thread, the four epilogue and the four builder warps
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // the first thread to give up stops the scan and marks every instance
  auto fail = [&]() {
    atomicExch(abort_flag, 1);
    if (atomicExch(a.abort, 1) == 0)
      for (int q = 0; q < a.count; ++q) atomicOr(a.inst[q].status, FQ_BIT_TIMEOUT);
  };

  if (warp == 0) {
    if (lane == 0) {  // ---------------- unit taker and TMA producer
      int g = 0;
      bool ok = true;
      // the next unit is taken one unit ahead, so that the atomic's round trip hides behind the
      // current unit's loads (units are still taken, and so processed, in increasing order)
      int u_next = (int)atomicAdd(a.next, 1u);
      for (int i = 0;; ++i) {
        const int slot = i % R;
        if (i >= R && !(ok = mbar_wait_or(uempty0 + 8 * slot, ((i / R) - 1) & 1, a.abort))) break;
        const bool stop = *(volatile int*)abort_flag || *(const volatile int*)a.abort;
        const ScanUnit d = stop ? ScanUnit{SU_END, 0, 0, 0, 0} : scan_decode(a, u_next);
        if (d.type != SU_END) u_next = (int)atomicAdd(a.next, 1u);
        volatile int* rs = ring + 5 * slot;
        rs[0] = d.type;
        rs[1] = d.inst;
        rs[2] = d.m;
        rs[3] = d.p;
        rs[4] = d.t;
        mbar_arrive(ufull0 + 8 * slot);  // release: the consumers read the slot after their wait
        if (d.type == SU_END) break;
        if (d.type != SU_TERM) continue;
        const ScanInst& I = a.inst[d.inst];
        const int tj = d.t / I.tiles_i, j0 = tj * BM, i0 = (d.t - tj * I.tiles_i) * BN;
        ok = scan_wait(I.omegacnt + (d.m & 1), 4u * I.nblk * (unsigned)(d.m / 2 + 1), a.abort);
        if (ok && d.p > 0)
          ok = scan_wait(I.termcnt + (size_t)(d.p - 1) * I.tiles_j + tj, 4u * I.tiles_i * (unsigned)(d.m + 1),
                         a.abort);
        if (ok && d.p == 0 && d.m > 0)
          ok = scan_wait(I.termcnt + (size_t)(I.L - 1) * I.tiles_j + tj, 4u * I.tiles_i * (unsigned)d.m, a.abort);
        if (!ok) break;
        fence_proxy_async_global();  // the epilogues' generic stores, before this thread's TMA reads
        const int av = ((d.m * (I.L & 1)) & 1) ^ (d.p & 1);
        const CUtensorMap* la = I.a[av];
        const CUtensorMap* ros = I.os[d.m & 1];
        const CUtensorMap* roa = I.oa[d.m & 1];
#pragma unroll
        for (int q = 0; q < NS; ++q) {  // the descriptors live in global memory: fetch them early
          asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)(la + q)) : "memory");
          asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)(ros + q)) : "memory");
          asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)(roa + q)) : "memory");
        }
        for (int kb = 0; kb < I.nk; ++kb) {
          const int s = g % STAGES;
          if (g >= STAGES && !(ok = mbar_wait_or(empty0 + 8 * s, ((g / STAGES) - 1) & 1, abort_flag))) break;
          const uint32_t st = base + s * Cfg::STAGE_BYTES;
          const uint32_t bar = full0 + 8 * s;
          mbar_expect_tx(bar, Cfg::STAGE_BYTES);
          const int kx = kb * BKE;
#pragma unroll
          for (int q = 0; q < NS; ++q) {
            tma_load_2d(st + q * Cfg::A_BYTES, &la[q], bar, kx, j0);
            tma_load_2d(st + (NS + q) * Cfg::A_BYTES, &la[q], bar, I.np + kx, j0);
            tma_load_2d(st + 2 * NS * Cfg::A_BYTES + q * Cfg::B_BYTES, &ros[q], bar, kx, i0);
            tma_load_2d(st + 2 * NS * Cfg::A_BYTES + (NS + q) * Cfg::B_BYTES, &roa[q], bar, kx, i0);
          }
          ++g;
        }
        if (!ok) break;
      }
      if (!ok) fail();
      // every copy issued must have landed before the CTA may exit
      for (int q = max(0, g - STAGES); q < g; ++q) mbar_wait(full0 + 8 * (q % STAGES), (q / STAGES) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ---------------- MMA issuer (as k_split_chain)
      constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                 ((uint32_t)(BM >> 4) << 24);
      constexpr uint32_t idesc_neg = idesc | (1u << 13);
      int g = 0, k = 0;
      bool ok = true;
      for (int i = 0;; ++i) {
        const int slot = i % R;
        if (!(ok = mbar_wait_or(ufull0 + 8 * slot, (i / R) & 1, abort_flag))) break;
        const int type = ring[5 * slot], inst = ring[5 * slot + 1];
        mbar_arrive(uempty0 + 8 * slot);
        if (type == SU_END) break;
        if (type != SU_TERM) continue;
        const int nk = a.inst[inst].nk;
        const int b = k & 1;
        if (k >= 2 && !(ok = mbar_wait_or(tempty0 + 8 * b, ((k >> 1) - 1) & 1, abort_flag))) break;
        const uint32_t acc = tmem + (uint32_t)b * BUF_COLS;
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = g % STAGES;
          if (!(ok = mbar_wait_or(full0 + 8 * s, (g / STAGES) & 1, abort_flag))) break;
          tc_fence_after();
          const uint32_t st = base + s * Cfg::STAGE_BYTES;
#pragma unroll
          for (int pp = 0; pp < Pairs<NS>::N; ++pp) {
            const uint32_t pr = st + Pairs<NS>::a(pp) * Cfg::A_BYTES;
            const uint32_t pi = st + (NS + Pairs<NS>::a(pp)) * Cfg::A_BYTES;
            const uint32_t os = st + 2 * NS * Cfg::A_BYTES + Pairs<NS>::b(pp) * Cfg::B_BYTES;
            const uint32_t oa = st + 2 * NS * Cfg::A_BYTES + (NS + Pairs<NS>::b(pp)) * Cfg::B_BYTES;
#pragma unroll
            for (int kk = 0; kk < BKE / 16; ++kk) {
              const uint32_t first = (kb == 0 && pp == 0 && kk == 0) ? 0u : 1u;
              const uint64_t dpr = smem_desc<Cfg::ROWB>(pr + 32 * kk), dpi = smem_desc<Cfg::ROWB>(pi + 32 * kk);
              const uint64_t dos = smem_desc<Cfg::ROWB>(os + 32 * kk), doa = smem_desc<Cfg::ROWB>(oa + 32 * kk);
              mma_bf16(acc, dpr, dos, idesc, first);
              mma_bf16(acc, dpi, doa, idesc_neg, 1u);
              mma_bf16(acc + BN, dpr, doa, idesc, first);
              mma_bf16(acc + BN, dpi, dos, idesc, 1u);
            }
          }
          mma_commit(empty0 + 8 * s);
        }
        if (!ok) break;
        mma_commit(tfull0 + 8 * b);
        ++k;
      }
      if (!ok) fail();
      mma_commit(done);  // every MMA issued above has completed once this arrives
      mbar_wait(done, 0);
    }
  } else if (warp < 6) {  // ---------------- epilogue warps 2-5: the term units' epilogues
    const int quarter = warp & 3;
    bool ok = true;
    int k = 0;
    for (int i = 0;; ++i) {
      const int slot = i % R;
      bool go = __all_sync(0xffffffffu, mbar_wait_or(ufull0 + 8 * slot, (i / R) & 1, abort_flag));
      if (!go) {
        ok = false;
        break;
      }
      const ScanUnit d{ring[5 * slot], ring[5 * slot + 1], ring[5 * slot + 2], ring[5 * slot + 3],
                       ring[5 * slot + 4]};
      __syncwarp();
      if (lane == 0) mbar_arrive(uempty0 + 8 * slot);
      if (d.type == SU_END) break;
      if (d.type != SU_TERM) continue;
      const ScanInst& I = a.inst[d.inst];
      // term unit
      const int b = k & 1;
      go = mbar_wait_or(tfull0 + 8 * b, (k >> 1) & 1, abort_flag);
      tc_fence_after();
      go = __all_sync(0xffffffffu, go);
      if (!go) {
        ok = false;
        break;
      }
      const int tj = d.t / I.tiles_i, j0 = tj * BM, i0 = (d.t - tj * I.tiles_i) * BN;
      // the previous term's outputs this epilogue reads were released with its counter
      if (d.p > 0) ld_acquire_u32(I.termcnt + (size_t)(d.p - 1) * I.tiles_j + tj);
      else if (d.m > 0) ld_acquire_u32(I.termcnt + (size_t)(I.L - 1) * I.tiles_j + tj);
      else ld_acquire_u32(I.omegacnt);  // the initial masters, written by the prologue's B units
      SplitEpi e;
      scan_epi(I, d.m, d.p, e);
      const int j = j0 + quarter * 32 + lane;
      const uint32_t trow = tmem + (uint32_t)b * BUF_COLS + ((uint32_t)(quarter * 32) << 16);
      bool bad = false;
      double dsr = 0.0, dsi = 0.0;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 16) {
        float yr[16], yi[16];
        tmem_ld16(trow + c0, yr);
        tmem_ld16(trow + BN + c0, yi);
        tmem_wait_ld();
        const int ib = i0 + c0;
        if (j >= e.nc || ib >= e.n) continue;
        epi_chunk<NS, EPI_FWD>(e, yr, yi, j, ib, bad, dsr, dsi);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty0 + 8 * b);
      if (bad) atomicOr(I.status, FQ_BIT_BOUND);
      // this warp's stores of the tile made visible (to the async proxy too), then one release per
      // warp: a state block is done when the four epilogue warps of each of its tiles have counted
      fence_proxy_async_global();
      __threadfence();
      __syncwarp();
      if (lane == 0) red_release_add(I.termcnt + (size_t)d.p * I.tiles_j + tj, 1u);
      ++k;
    }
    if (!ok) fail();
  } else {  // ---------------- builder warps 6-9: the B and W units
    const int tid = threadIdx.x - 192;
    bool ok = true;
    for (int i = 0;; ++i) {
      const int slot = i % R;
      if (!__all_sync(0xffffffffu, mbar_wait_or(ufull0 + 8 * slot, (i / R) & 1, abort_flag))) {
        ok = false;
        break;
      }
      const ScanUnit d{ring[5 * slot], ring[5 * slot + 1], ring[5 * slot + 2], ring[5 * slot + 3],
                       ring[5 * slot + 4]};
      __syncwarp();
      if (lane == 0) mbar_arrive(uempty0 + 8 * slot);
      if (d.type == SU_END) break;
      if (d.type == SU_TERM) continue;
      const ScanInst& I = a.inst[d.inst];
      if (d.type == SU_OMEGA) {
        if (d.m >= I.steps) continue;  // the step after the last one
        if (d.m >= 2) {  // buffer m & 1 was read by step m - 2: wait until it has finished everywhere
          bool w = true;
          for (int tj = lane; tj < I.tiles_j && w; tj += 32)
            w = scan_wait(I.termcnt + (size_t)(I.L - 1) * I.tiles_j + tj, 4u * I.tiles_i * (unsigned)(d.m - 1),
                          a.abort);
          if (!__all_sync(0xffffffffu, w)) {
            ok = false;
            break;
          }
        }
        scan_omega_rows<NS>(I, d.m, d.t * BLOCK_ROWS, tid);
        fence_proxy_async_global();  // these generic stores, before the TMA reads of later units
        __threadfence();
        __syncwarp();
        if (lane == 0) red_release_add(I.omegacnt + (d.m & 1), 1u);
        continue;
      }
      if (d.type == SU_STORE) {
        const int j0 = d.t * BLOCK_ROWS;
        if (!__all_sync(0xffffffffu, scan_wait(I.termcnt + (size_t)(I.L - 1) * I.tiles_j + j0 / BM,
                                                4u * I.tiles_i * (unsigned)I.steps, a.abort))) {
          ok = false;
          break;
        }
        scan_store_rows(I, j0, tid);
        continue;
      }
    }
    if (!ok) fail();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

int scan_ns(const fq_plan* p) { return p->precision == FQ_BF16X6 ? 3 : 2; }

// Tile width of the scan: the one the plans' (autotuned) widths favour, weighted by their work.
int scan_bn(fq_plan* const* plans, int count) {
  double w128 = 0, w64 = 0;
  for (int i = 0; i < count; ++i) {
    const double c = (double)plans[i]->n * plans[i]->n * plans[i]->n * plans[i]->steps * plans[i]->L;
    (plans[i]->tile_n == 128 ? w128 : w64) += c;
  }
  return w128 >= w64 ? 128 : 64;
}

// Layout of the scan's own region (after the plans' workspaces): instance table, segment table,
// counters (one memset clears them), then per instance the second pair of Omega~ slice buffers.
struct ScanLayout {
  size_t inst, seg, cnt, cnt_words, total;
  std::vector<size_t> omega2;        // per instance: offset of os_buf[1] (oa_buf[1] follows)
  std::vector<size_t> termcnt;       // per instance: word offset of its counters in cnt
  std::vector<ScanSeg> segs;
  int npro = 0, nstep = 0, nend = 0, upro = 0, ustep = 0, uend = 0;
};

// What the unit table needs of an instance: N, the series length L and the slices per operand.
struct ScanShape {
  int n, L, ns;
};

int np_of(int n) { return (n + 127) & ~127; }
int tiles_j_of(int n) { return (n + BM - 1) / BM; }

std::vector<ScanShape> shapes_of(fq_plan* const* plans, int count) {
  std::vector<ScanShape> sh(count);
  for (int i = 0; i < count; ++i) sh[i] = ScanShape{plans[i]->n, plans[i]->L, scan_ns(plans[i])};
  return sh;
}

// The unit table and the scan's region; false when the unit count would not fit the 32-bit counter.
// Step order: term p of every instance (costliest first, state-block-major inside a term) before
// term p + 1 of any, each instance's Omega~ blocks of the next step in L - 1 shares after its terms
// 1 .. L - 1 (after term 0 when L = 1), so the builder warps' work spreads over the step.
bool scan_layout(const std::vector<ScanShape>& sh, int steps, int bn, ScanLayout& L) {
  const int count = (int)sh.size();
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return (double)sh[x].n * sh[x].n * sh[x].n * sh[x].L > (double)sh[y].n * sh[y].n * sh[y].n * sh[y].L;
  });
  long long u = 0;
  L.segs.clear();
  for (int i : order) {  // prologue: B(i, 0, *)
    L.segs.push_back(ScanSeg{(int)u, SU_OMEGA, i, 0});
    u += np_of(sh[i].n) / BLOCK_ROWS;
  }
  L.npro = (int)L.segs.size();
  L.upro = (int)u;
  u = 0;
  int lmax = 0;
  for (const ScanShape& q : sh) lmax = std::max(lmax, q.L);
  for (int p = 0; p < lmax; ++p)
    for (int i : order) {
      const ScanShape& q = sh[i];
      if (p >= q.L) continue;
      L.segs.push_back(ScanSeg{(int)u, SU_TERM, i, p});
      u += (long long)(np_of(q.n) / bn) * tiles_j_of(q.n);
      const int shares = std::max(1, q.L - 1), c = std::max(0, p - 1), nb = np_of(q.n) / BLOCK_ROWS;
      if (p >= std::min(1, q.L - 1)) {
        const int b0 = (int)((long long)c * nb / shares), b1 = (int)((long long)(c + 1) * nb / shares);
        if (b1 > b0) L.segs.push_back(ScanSeg{(int)u, SU_OMEGA, i, b0});
        u += b1 - b0;
      }
      if (u > INT_MAX / 4) return false;
    }
  L.nstep = (int)L.segs.size() - L.npro;
  L.ustep = (int)u;
  u = 0;
  for (int i : order) {
    L.segs.push_back(ScanSeg{(int)u, SU_STORE, i, 0});
    u += (sh[i].n + BLOCK_ROWS - 1) / BLOCK_ROWS;
  }
  L.nend = (int)L.segs.size() - L.npro - L.nstep;
  L.uend = (int)u;
  if ((long long)L.upro + (long long)steps * L.ustep + L.uend > INT_MAX - 4096) return false;
  size_t off = 0;
  L.inst = off;
  off += up256(sizeof(ScanInst) * count);
  L.seg = off;
  off += up256(sizeof(ScanSeg) * L.segs.size());
  L.termcnt.resize(count);
  size_t words = 2;  // next, abort
  for (int i = 0; i < count; ++i) {
    L.termcnt[i] = words;
    words += (size_t)sh[i].L * tiles_j_of(sh[i].n) + 2;
  }
  L.cnt = off;
  L.cnt_words = words;
  off += up256(sizeof(unsigned int) * words);
  L.omega2.resize(count);
  for (int i = 0; i < count; ++i) {
    const size_t slices = (size_t)sh[i].ns * np_of(sh[i].n) * np_of(sh[i].n);
    L.omega2[i] = off;
    off += 2 * up256(sizeof(__nv_bfloat16) * slices);
  }
  L.total = off;
  return true;
}

template <int NS, int BN, int BKE>
fq_status scan_capture(fq_plan* const* plans, int count, void* const* d_U, char* ws, const size_t* off, char* extra,
                       ScanLayout& lay, cudaGraph_t* graph) {
  fq_status st = encode_fn();
  if (st != FQ_OK) return st;
  std::vector<ScanInst> inst(count);
  for (int i = 0; i < count; ++i) {
    fq_plan* p = plans[i];
    SplitWs w;
    fq_split_workspace(p, p->n, ws + off[i], &w);
    ScanInst& I = inst[i];
    I = ScanInst{};
    I.n = p->n;
    I.np = w.np;
    I.kp = w.kp;
    I.ldm = w.ldm;
    I.L = p->L;
    I.steps = p->steps;
    I.tiles_i = w.np / BN;
    I.tiles_j = tiles_j_of(p->n);
    I.nk = (p->n + BKE - 1) / BKE;  // the operands' columns beyond N are zero
    I.nblk = w.np / BLOCK_ROWS;
    I.bstride = w.bstride;
    I.astride = w.astride;
    I.h0 = p->d_h0;
    I.h1 = p->d_h1;
    I.k = p->d_k;
    I.scal = p->d_scal;
    I.sbeta = p->sbeta;
    I.ph_re = p->phase_re;
    I.ph_im = p->phase_im;
    for (int l = 0; l <= p->L; ++l) I.cheb[l] = p->cheb[l];
    I.status = p->d_status;
    I.u = (double2*)d_U[i];
    I.os_buf[0] = w.os;
    I.oa_buf[0] = w.oa;
    I.os_buf[1] = (__nv_bfloat16*)(extra + lay.omega2[i]);
    I.oa_buf[1] = (__nv_bfloat16*)(extra + lay.omega2[i] + up256(sizeof(__nv_bfloat16) * NS * w.bstride));
    for (int v = 0; v < 2; ++v) I.abuf[v] = w.a[v];
    for (int q = 0; q < 3; ++q)
      for (int r = 0; r < 2; ++r) I.m[q][r] = w.m[q][r];
    unsigned int* cnt = (unsigned int*)(extra + lay.cnt);
    I.termcnt = cnt + lay.termcnt[i];
    I.omegacnt = I.termcnt + (size_t)p->L * I.tiles_j;
    for (int v = 0; v < 2; ++v)
      for (int q = 0; q < NS; ++q) {
        if ((st = make_map(&I.a[v][q], w.a[v] + q * w.astride, w.ncp, w.kp, BM, BKE)) != FQ_OK) return st;
        if ((st = make_map(&I.os[v][q], I.os_buf[v] + q * w.bstride, w.np, w.np, BN, BKE)) != FQ_OK) return st;
        if ((st = make_map(&I.oa[v][q], I.oa_buf[v] + q * w.bstride, w.np, w.np, BN, BKE)) != FQ_OK) return st;
      }
  }
  // the tables are written once, before the capture: the graph only clears the counters
  cudaError_t e = cudaMemcpy(extra + lay.inst, inst.data(), sizeof(ScanInst) * count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(extra + lay.seg, lay.segs.data(), sizeof(ScanSeg) * lay.segs.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fq_cuda_fail(e, "scan tables");
  static std::atomic<unsigned> attr_set{0};
  if (fq_first_on_device(attr_set)) {
    e = cudaFuncSetAttribute(k_split_scan<NS, BN, BKE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)ScanCfg<NS, BN, BKE>::SMEM);
    if (e != cudaSuccess) return fq_cuda_fail(e, "scan kernel shared-memory attribute");
  }
  ScanArgs args{};
  args.inst = (const ScanInst*)(extra + lay.inst);
  args.seg = (const ScanSeg*)(extra + lay.seg);
  args.npro = lay.npro;
  args.nstep = lay.nstep;
  args.nend = lay.nend;
  args.upro = lay.upro;
  args.ustep = lay.ustep;
  args.uend = lay.uend;
  args.steps = plans[0]->steps;
  args.count = count;
  args.total = lay.upro + args.steps * lay.ustep + lay.uend;
  unsigned int* cnt = (unsigned int*)(extra + lay.cnt);
  args.next = cnt;
  args.abort = (int*)(cnt + 1);
  cudaStream_t s = nullptr;
  e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) return fq_cuda_fail(e, "scan stream");
  e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaMemsetAsync(cnt, 0, sizeof(unsigned int) * lay.cnt_words, s);
    k_split_scan<NS, BN, BKE><<<fq_sm_count(), SCAN_THREADS, ScanCfg<NS, BN, BKE>::SMEM, s>>>(args);
    cudaError_t le = cudaGetLastError();
    e = cudaStreamEndCapture(s, graph);
    if (le != cudaSuccess) e = le;
  }
  cudaStreamDestroy(s);
  return e == cudaSuccess ? FQ_OK : fq_cuda_fail(e, "scan capture");
}

}  // namespace

int fq_scan_eligible(fq_plan* const* plans, int count) {
  if (!plans || count < 1 || !plans[0]) return 0;
  for (int i = 0; i < count; ++i) {
    const fq_plan* p = plans[i];
    if (!p || p->path != PATH_DENSE_SPLIT || p->order != 4 || p->precision != plans[0]->precision ||
        p->steps != plans[0]->steps || p->L < 1 || p->L > SCAN_MAXL || p->n < 1)
      return 0;
  }
  ScanLayout lay;
  return scan_layout(shapes_of(plans, count), plans[0]->steps, scan_bn(plans, count), lay) ? 1 : 0;
}

size_t fq_scan_extra_bytes(fq_plan* const* plans, int count) {
  if (!fq_scan_eligible(plans, count)) return 0;
  ScanLayout lay;
  scan_layout(shapes_of(plans, count), plans[0]->steps, scan_bn(plans, count), lay);
  return lay.total;
}

fq_status fq_scan_graph(fq_plan* const* plans, int count, void* const* d_U, void* ws, const size_t* off,
                        size_t extra_off, cudaGraph_t* graph) {
  if (!fq_scan_eligible(plans, count)) {
    fq_set_error("batched scan: every plan must be a split-precision (BF16X3 or BF16X6) dense plan of order 4 with "
                 "the same precision and step count, and L <= %d",
                 SCAN_MAXL);
    return FQ_EUNSUPPORTED;
  }
  const int bn = scan_bn(plans, count);
  ScanLayout lay;
  scan_layout(shapes_of(plans, count), plans[0]->steps, bn, lay);
  char* base = (char*)ws;
  char* extra = base + extra_off;
  const bool x6 = plans[0]->precision == FQ_BF16X6;
  if (x6)
    return bn == 128 ? scan_capture<3, 128, 32>(plans, count, d_U, base, off, extra, lay, graph)
                     : scan_capture<3, 64, 32>(plans, count, d_U, base, off, extra, lay, graph);
  return bn == 128 ? scan_capture<2, 128, 32>(plans, count, d_U, base, off, extra, lay, graph)
                   : scan_capture<2, 64, 64>(plans, count, d_U, base, off, extra, lay, graph);
}

// Test hook, outside the public header: the unit table of a scan of `count` instances (sizes n[i],
// series lengths L[i]) over `steps` steps with tiles of bn rows of Omega~, as (begin, type, instance,
// p) quadruples in seg (capacity cap quadruples): prologue, one step, end; counts receives the
// segments and units of each part [npro, nstep, nend, upro, ustep, uend].  Returns the number of
// segments, or -1 (arguments, capacity, or a unit count past the 32-bit counter).  Host only.
extern "C" int fq_scan_table(int count, const int* n, const int* L, int steps, int bn, int* seg, int cap,
                             int* counts) {
  if (count < 1 || !n || !L || !seg || !counts || steps < 1 || (bn != 64 && bn != 128)) return -1;
  std::vector<ScanShape> sh(count);
  for (int i = 0; i < count; ++i) {
    if (n[i] < 1 || L[i] < 1 || L[i] > SCAN_MAXL) return -1;
    sh[i] = ScanShape{n[i], L[i], 2};
  }
  ScanLayout lay;
  if (!scan_layout(sh, steps, bn, lay) || (int)lay.segs.size() > cap) return -1;
  for (size_t k = 0; k < lay.segs.size(); ++k) {
    seg[4 * k] = lay.segs[k].begin;
    seg[4 * k + 1] = lay.segs[k].type;
    seg[4 * k + 2] = lay.segs[k].inst;
    seg[4 * k + 3] = lay.segs[k].p;
  }
  const int c[6] = {lay.npro, lay.nstep, lay.nend, lay.upro, lay.ustep, lay.uend};
  for (int k = 0; k < 6; ++k) counts[k] = c[k];
  return (int)lay.segs.size();
}
