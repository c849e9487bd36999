// Split-precision dense GEMM core on the 5th-generation tensor cores (tcgen05, sm_103a), shared by
// the forward Chebyshev chain (dense_split.cu) and the adjoint (adjoint_split.cu).
//
// One product on a block of state rows: Y^T = Psi^T Omega~^T with Omega~ = S + i A (S real
// symmetric, A real antisymmetric), i.e. with X.B := sum_k X[j][k] B[i][k]
//   Yr = Psi_r.S - Psi_i.A,   Yi = Psi_r.A + Psi_i.S       (HAS_A; A = 0 drops two streams).
// Each K stage loads the Psi_r, Psi_i tiles and one S (and one A) tile, and four MMA streams
// (the minus sign through the instruction's negate-A bit) use every tile twice.  Every operand
// is held as NS BF16 slices (x = x_0 + x_1 + ..., x_s = bf16 of the remainder), and the products
// x_a y_b with a + b < NS (3 for NS = 2, 6 for NS = 3) are summed in FP32 in tensor memory.
// The epilogue (epi_chunk) is one of: the Chebyshev term (recurrence psi_{l+1} = -2i Y +
// psi_{l-1}, Bessel accumulation and step phase on FP32 masters, Eqs. 10 and 12), the adjoint
// term, or the gradient dot; the first two also write the next product's slices.
//
// k_split_term: one 128-row x BN-column tile per CTA of 128 threads.  k_split_persist: one CTA
// per SM walks its tiles with a dedicated TMA warp, MMA warp and four epilogue warps, and two
// tensor-memory buffers so that a tile's epilogue overlaps the next tile's MMAs.  Tiles are
// rasterized in groups of 8 row blocks so that co-running CTAs share operands in L2.  TMA loads
// are K-major with 128- or 64-byte swizzle; stages and buffers are handed over by mbarriers.
// Every wait is bounded; a wait that gives up records FQ_BIT_TIMEOUT, drains this CTA's own
// copies and MMAs, frees tensor memory and returns.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "internal.h"

namespace {


constexpr int BM = 128;      // state rows per tile (tcgen05 M)
constexpr int NTHREADS = 128;
constexpr int RASTER_GROUP = 8;
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

// ------------------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false if the phase did not complete within kWaitCycles.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          dst),
      "l"((uint64_t)map), "r"(bar), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor: K-major rows of ROWB bytes (128 or 64) with the matching
// swizzle, 8-row atoms of 8 * ROWB bytes.
template <int ROWB>
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);           // start address
  d |= (uint64_t)1 << 16;                             // leading-dimension offset (unused, swizzled K-major)
  d |= (uint64_t)((8 * ROWB) >> 4) << 32;             // stride between 8-row atoms
  d |= (uint64_t)1 << 46;                             // descriptor version for tcgen05
  d |= (uint64_t)(ROWB == 128 ? 2 : 4) << 61;         // 128-byte or 64-byte swizzle
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// ------------------------------------------------------------------------- slices
template <int NS>
__device__ __forceinline__ void split_f32(float x, __nv_bfloat16 (&s)[NS]) {
  float r = x;
#pragma unroll
  for (int q = 0; q < NS; ++q) {
    s[q] = __float2bfloat16_rn(r);
    r -= __bfloat162float(s[q]);
  }
}

template <int NS>
__device__ __forceinline__ void split_f64(double x, __nv_bfloat16 (&s)[NS]) {
  double r = x;
#pragma unroll
  for (int q = 0; q < NS; ++q) {
    s[q] = __double2bfloat16(r);
    r -= (double)__bfloat162float(s[q]);
  }
}

// Entry (i, c) of Omega~_m = S + i A with S = sa H0 + sb H1 - sbeta 1 and A = sc [H0, H1]
// (Eqs. 11 and 14), formed in FP32 from the FP64 operators: the split paths keep at most 24 bits
// of an entry (three BF16 slices), and FP64 arithmetic runs at a small fraction of the FP32 rate
// on this GPU.  The multiply-adds are spelt out so that every kernel forming it rounds alike.
__device__ __forceinline__ void omega_entry(double h0, double h1, double k, bool diag, float sa, float sb,
                                            float sc, float sbeta, float& S, float& A) {
  S = fmaf(sa, (float)h0, fmaf(sb, (float)h1, diag ? -sbeta : 0.f));
  A = sc * (float)k;
}

// Left operand and FP32 masters of the initial block: identity rows (build_UT) or given states.
template <int NS>
__global__ void k_split_init(const double2* __restrict__ x0, int n, int nc, int ldm, int np, int kp, float* mre,
                             float* mim, __nv_bfloat16* sl, size_t slice_stride) {
  const size_t total = (size_t)nc * kp;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(q / kp), c = (int)(q % kp);
    const bool im_half = c >= np;
    const int i = im_half ? c - np : c;
    float v = 0.f;
    if (i < n) {
      double2 z = x0 ? x0[(size_t)j * n + i] : make_double2(i == j ? 1.0 : 0.0, 0.0);
      v = (float)(im_half ? z.y : z.x);
      if (im_half) mim[(size_t)j * ldm + i] = v;
      else mre[(size_t)j * ldm + i] = v;
    }
    __nv_bfloat16 s[NS];
    split_f32<NS>(v, s);
#pragma unroll
    for (int t = 0; t < NS; ++t) sl[t * slice_stride + q] = s[t];
  }
}

// Products kept for NS slices: (a, b) with a + b < NS, ordered smallest first.
template <int NS> struct Pairs;
template <> struct Pairs<2> {
  static constexpr int N = 3;
  static __device__ __forceinline__ int a(int p) { return p == 0 ? 1 : 0; }  // (1,0), (0,1), (0,0)
  static __device__ __forceinline__ int b(int p) { return p == 1 ? 1 : 0; }
};
template <> struct Pairs<3> {
  static constexpr int N = 6;
  static __device__ __forceinline__ int a(int p) { const int t[6] = {1, 0, 2, 1, 0, 0}; return t[p]; }
  static __device__ __forceinline__ int b(int p) { const int t[6] = {1, 2, 0, 0, 1, 0}; return t[p]; }
};

// Workspace of the split chain (dense_split.cu's fq_split_workspace): the right operand's slices
// (S, A), two left-operand slice buffers (ping-pong across terms), three FP32 master state buffers
// (planar) for psi_l / psi_{l-1} / acc, and the chain counters.
struct SplitWs {
  __nv_bfloat16* os;  // S slices
  __nv_bfloat16* oa;  // A slices
  __nv_bfloat16* a[2];
  float* m[3][2];
  unsigned int* flags;  // chain counters: [CHAIN_MAXP][row blocks]
  int np, kp, ldm, ncp;
  size_t bstride, astride;
};

struct SplitMaps {
  CUtensorMap a[3];   // left operand slices [ncp][2 Np]: Psi_r in columns [0, Np), Psi_i in [Np, 2 Np)
  CUtensorMap os[3];  // S slices [Np][Np]
  CUtensorMap oa[3];  // A slices [Np][Np]
};

// Epilogue of one split GEMM (Y = left . right^T on a 128 x BN tile, FP32 in tensor memory).
enum SplitMode {
  EPI_FWD = 0,  // Chebyshev term: psi_{l+1} = -2i Y + psi_{l-1}, acc += a psi_{l+1}, phase at the last term
  EPI_ADJ = 1,  // adjoint term: out = cpa g + i cw Y + b2
  EPI_DOT = 2,  // gradient dot: partial[cta] = sum over the tile of conj(b) Y
};

struct SplitEpi {
  int n, nc, ldm, np;          // dims; ldm: FP32 master row stride; np: real part width in K'
  const float* cur_re;         // FWD: psi_l masters (first term: psi_0); ADJ: g; DOT: b
  const float* cur_im;
  const float* prev_re;        // FWD: psi_{l-1}; ADJ: b2 (NULL: absent)
  const float* prev_im;
  float* acc_re;
  float* acc_im;
  float* out_re;               // FWD: psi_{l+1} (in place of psi_{l-1}) or X at the last term; ADJ: out
  float* out_im;
  __nv_bfloat16* slice_out;    // next left operand: NS slices, each [nc][Kp]
  size_t slice_stride;         // elements between slices
  int kp;
  float cpa_re, cpa_im, cw;    // ADJ coefficients
  double2* partial;            // DOT output, one per CTA
  fq_term t;
};

template <int NS, int BN, int BKE, bool HAS_A>
struct SplitCfg {
  static constexpr int ROWB = BKE * 2;                // bytes per K row of a stage (swizzle span)
  static constexpr int A_BYTES = BM * ROWB;           // one slice of Psi_r or Psi_i, one stage
  static constexpr int B_BYTES = BN * ROWB;           // one slice of S or A, one stage
  static constexpr int STAGE_BYTES = 2 * NS * A_BYTES + (HAS_A ? 2 : 1) * NS * B_BYTES;
  static constexpr int STAGES = (215040 / STAGE_BYTES) > 4 ? 4 : (215040 / STAGE_BYTES);
  static constexpr int TMEM_COLS = 2 * BN <= 32 ? 32 : (2 * BN <= 64 ? 64 : (2 * BN <= 128 ? 128 : 256));
  static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 1024 + 256;
};

__device__ __forceinline__ void store_f4(float* p, const float* v) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void load_f4(const float* p, float* v) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}

// Loads cnt (<= 16) FP32 entries at p + idx (zero beyond cnt; all zero when p is NULL).
__device__ __forceinline__ void load16(const float* p, size_t idx, int cnt, float (&v)[16]) {
  if (p && cnt == 16) {
#pragma unroll
    for (int q = 0; q < 16; q += 4) load_f4(p + idx + q, v + q);
  } else {
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = (p && q < cnt) ? p[idx + q] : 0.f;
  }
}

__device__ __forceinline__ void store16(float* p, size_t idx, int cnt, const float (&v)[16]) {
  if (cnt == 16) {
#pragma unroll
    for (int q = 0; q < 16; q += 4) store_f4(p + idx + q, v + q);
  } else {
#pragma unroll
    for (int q = 0; q < 16; ++q)
      if (q < cnt) p[idx + q] = v[q];
  }
}

// NS BF16 slices of 16 new complex entries into the next left operand (row j, columns ib..ib+cnt):
// the real parts at column ib, the imaginary parts at column np + ib of each slice.
template <int NS>
__device__ __forceinline__ void store_slices(const SplitEpi& e, int j, int ib, int cnt, const float (&o_r)[16],
                                             const float (&o_i)[16]) {
  uint32_t wre[NS][8], wim[NS][8];  // two bf16 per word, element 2w in the low half
#pragma unroll
  for (int q = 0; q < 16; q += 2) {
    __nv_bfloat16 r0[NS], r1[NS], m0[NS], m1[NS];
    split_f32<NS>(o_r[q], r0);
    split_f32<NS>(o_r[q + 1], r1);
    split_f32<NS>(o_i[q], m0);
    split_f32<NS>(o_i[q + 1], m1);
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      wre[t][q / 2] = (uint32_t)__bfloat16_as_ushort(r0[t]) | ((uint32_t)__bfloat16_as_ushort(r1[t]) << 16);
      wim[t][q / 2] = (uint32_t)__bfloat16_as_ushort(m0[t]) | ((uint32_t)__bfloat16_as_ushort(m1[t]) << 16);
    }
  }
  const size_t srow = (size_t)j * e.kp + ib;
  if (cnt == 16) {
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      uint4* dr = reinterpret_cast<uint4*>(e.slice_out + t * e.slice_stride + srow);
      uint4* di = reinterpret_cast<uint4*>(e.slice_out + t * e.slice_stride + srow + e.np);
      dr[0] = make_uint4(wre[t][0], wre[t][1], wre[t][2], wre[t][3]);
      dr[1] = make_uint4(wre[t][4], wre[t][5], wre[t][6], wre[t][7]);
      di[0] = make_uint4(wim[t][0], wim[t][1], wim[t][2], wim[t][3]);
      di[1] = make_uint4(wim[t][4], wim[t][5], wim[t][6], wim[t][7]);
    }
  } else {
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      if (q < cnt) {
#pragma unroll
        for (int t = 0; t < NS; ++t) {
          const uint32_t wr = wre[t][q / 2] >> (16 * (q & 1)), wi = wim[t][q / 2] >> (16 * (q & 1));
          e.slice_out[t * e.slice_stride + srow + q] = __ushort_as_bfloat16((unsigned short)(wr & 0xFFFFu));
          e.slice_out[t * e.slice_stride + srow + e.np + q] = __ushort_as_bfloat16((unsigned short)(wi & 0xFFFFu));
        }
      }
    }
  }
}

// Epilogue of one 16-column chunk of row j: Y entries yr, yi of columns ib .. ib + 15 (cnt valid).
template <int NS, int EPI>
__device__ __forceinline__ void epi_chunk(const SplitEpi& e, const float (&yr)[16], const float (&yi)[16], int j,
                                          int ib, bool& bad, double& dsr, double& dsi) {
  const float c0f = (float)e.t.coef0, cf = (float)e.t.coef, pr_ = (float)e.t.ph_re, pi_ = (float)e.t.ph_im;
  const float b2 = (float)e.t.bound2;
  const int cnt = min(16, e.n - ib);
  const size_t idx = (size_t)j * e.ldm + ib;
  if (EPI == EPI_DOT) {
    float br[16], bi[16];
    load16(e.cur_re, idx, cnt, br);
    load16(e.cur_im, idx, cnt, bi);
    float sr = 0.f, si = 0.f;
#pragma unroll
    for (int q = 0; q < 16; ++q) {  // conj(b) Y; entries beyond cnt are zero in b
      sr = fmaf(br[q], yr[q], fmaf(bi[q], yi[q], sr));
      si = fmaf(br[q], yi[q], fmaf(-bi[q], yr[q], si));
    }
    dsr += (double)sr;
    dsi += (double)si;
    return;
  }
  float o_r[16], o_i[16];
  if (EPI == EPI_ADJ) {  // out = cpa g + i cw Y + b2
    float g_r[16], g_i[16], p_r[16], p_i[16];
    load16(e.cur_re, idx, cnt, g_r);
    load16(e.cur_im, idx, cnt, g_i);
    load16(e.prev_re, idx, cnt, p_r);
    load16(e.prev_im, idx, cnt, p_i);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      o_r[q] = e.cpa_re * g_r[q] - e.cpa_im * g_i[q] - e.cw * yi[q] + p_r[q];
      o_i[q] = e.cpa_re * g_i[q] + e.cpa_im * g_r[q] + e.cw * yr[q] + p_i[q];
      bad |= q < cnt && !(o_r[q] * o_r[q] + o_i[q] * o_i[q] <= b2);
    }
    store16(e.out_re, idx, cnt, o_r);
    store16(e.out_im, idx, cnt, o_i);
    store_slices<NS>(e, j, ib, cnt, o_r, o_i);
    return;
  }
  // EPI_FWD
  float a_r[16], a_i[16], p_r[16], p_i[16];
  load16(e.t.first ? e.cur_re : e.prev_re, idx, cnt, p_r);
  load16(e.t.first ? e.cur_im : e.prev_im, idx, cnt, p_i);
  load16(e.t.first ? nullptr : e.acc_re, idx, cnt, a_r);
  load16(e.t.first ? nullptr : e.acc_im, idx, cnt, a_i);
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    float nr, ni, sr, si;
    if (e.t.first) {  // psi_1 = -i Y, acc = a_0 psi_0 + a_1 psi_1
      nr = yi[q];
      ni = -yr[q];
      sr = c0f * p_r[q] + cf * nr;
      si = c0f * p_i[q] + cf * ni;
    } else {  // psi_{l+1} = -2i Y + psi_{l-1}, acc += a_{l+1} psi_{l+1}
      nr = 2.f * yi[q] + p_r[q];
      ni = -2.f * yr[q] + p_i[q];
      sr = a_r[q] + cf * nr;
      si = a_i[q] + cf * ni;
    }
    bad |= q < cnt && !(nr * nr + ni * ni <= b2);
    if (e.t.last) {  // X = e^{-i beta h} (acc + a_L psi_L)
      o_r[q] = pr_ * sr - pi_ * si;
      o_i[q] = pr_ * si + pi_ * sr;
    } else {
      o_r[q] = nr;
      o_i[q] = ni;
    }
    a_r[q] = sr;
    a_i[q] = si;
  }
  store16(e.out_re, idx, cnt, o_r);
  store16(e.out_im, idx, cnt, o_i);
  if (!e.t.last) {
    store16(e.acc_re, idx, cnt, a_r);
    store16(e.acc_im, idx, cnt, a_i);
  }
  store_slices<NS>(e, j, ib, cnt, o_r, o_i);
}

// One split GEMM on a 128-row x BN-column tile of Y = left . right^T:
//   HAS_A:  Yr = Psi_r.S - Psi_i.A,  Yi = Psi_r.A + Psi_i.S   (right = S + i A)
//   !HAS_A: Yr = Psi_r.S,            Yi = Psi_i.S             (right = S real)
// followed by the epilogue EPI.
template <int NS, int BN, int BKE, int EPI, bool HAS_A>
__global__ void __launch_bounds__(NTHREADS, 1)
k_split_term(const __grid_constant__ SplitMaps maps, int nk, int tiles_j, int tiles_i, SplitEpi e) {
  using Cfg = SplitCfg<NS, BN, BKE, HAS_A>;
  constexpr int STAGES = Cfg::STAGES;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned stage buffers (swizzle atoms), then barriers
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = smem_raw + (base - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + STAGES * Cfg::STAGE_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  double* red = reinterpret_cast<double*>(gbase + STAGES * Cfg::STAGE_BYTES + 128);  // DOT: 4 warps x 2
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES), done = smem_u32(bars + 2 * STAGES);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // grouped rasterization: RASTER_GROUP row blocks sweep the column blocks together
  int tj, ti;
  {
    const int b = blockIdx.x, per = RASTER_GROUP * tiles_i, g = b / per;
    const int gj = min(RASTER_GROUP, tiles_j - g * RASTER_GROUP), r = b - g * per;
    tj = g * RASTER_GROUP + r % gj;
    ti = r / gj;
  }
  const int j0 = tj * BM, i0 = ti * BN;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"((uint32_t)Cfg::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    int issued = 0;
    bool ok = true;
    for (int kb = 0; kb < nk && ok; ++kb) {
      const int s = kb % STAGES;
      if (kb >= STAGES) {
        ok = mbar_wait(empty0 + 8 * s, ((kb / STAGES) - 1) & 1);
        if (!ok) break;
      }
      const uint32_t st = base + s * Cfg::STAGE_BYTES;
      const uint32_t bar = full0 + 8 * s;
      mbar_expect_tx(bar, Cfg::STAGE_BYTES);
      const int kx = kb * BKE;
#pragma unroll
      for (int q = 0; q < NS; ++q) {
        tma_load_2d(st + q * Cfg::A_BYTES, &maps.a[q], bar, kx, j0);                       // Psi_r
        tma_load_2d(st + (NS + q) * Cfg::A_BYTES, &maps.a[q], bar, e.np + kx, j0);         // Psi_i
        tma_load_2d(st + 2 * NS * Cfg::A_BYTES + q * Cfg::B_BYTES, &maps.os[q], bar, kx, i0);  // S
        if (HAS_A)
          tma_load_2d(st + 2 * NS * Cfg::A_BYTES + (NS + q) * Cfg::B_BYTES, &maps.oa[q], bar, kx, i0);  // A
      }
      issued = kb + 1;
    }
    if (!ok) {
      atomicExch(abort_flag, 1);
      atomicOr(e.t.status, FQ_BIT_TIMEOUT);
    }
    // drain: every copy this thread issued must have landed before the CTA may exit
    for (int kb = max(0, issued - STAGES); kb < issued; ++kb) mbar_wait(full0 + 8 * (kb % STAGES), (kb / STAGES) & 1);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                               ((uint32_t)(BM >> 4) << 24);
    constexpr uint32_t idesc_neg = idesc | (1u << 13);  // negate the left operand
    bool ok = true;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      ok = mbar_wait(full0 + 8 * s, (kb / STAGES) & 1);
      if (!ok || *(volatile int*)abort_flag) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t st = base + s * Cfg::STAGE_BYTES;
#pragma unroll
      for (int p = 0; p < Pairs<NS>::N; ++p) {
        const uint32_t pr = st + Pairs<NS>::a(p) * Cfg::A_BYTES;
        const uint32_t pi = st + (NS + Pairs<NS>::a(p)) * Cfg::A_BYTES;
        const uint32_t os = st + 2 * NS * Cfg::A_BYTES + Pairs<NS>::b(p) * Cfg::B_BYTES;
        const uint32_t oa = st + 2 * NS * Cfg::A_BYTES + (NS + Pairs<NS>::b(p)) * Cfg::B_BYTES;
#pragma unroll
        for (int kk = 0; kk < BKE / 16; ++kk) {
          const uint32_t first = (kb == 0 && p == 0 && kk == 0) ? 0u : 1u;
          const uint64_t dpr = smem_desc<Cfg::ROWB>(pr + 32 * kk), dpi = smem_desc<Cfg::ROWB>(pi + 32 * kk);
          const uint64_t dos = smem_desc<Cfg::ROWB>(os + 32 * kk);
          if (HAS_A) {
            const uint64_t doa = smem_desc<Cfg::ROWB>(oa + 32 * kk);
            mma_bf16(tmem, dpr, dos, idesc, first);
            mma_bf16(tmem, dpi, doa, idesc_neg, 1u);
            mma_bf16(tmem + BN, dpr, doa, idesc, first);
            mma_bf16(tmem + BN, dpi, dos, idesc, 1u);
          } else {
            mma_bf16(tmem, dpr, dos, idesc, first);
            mma_bf16(tmem + BN, dpi, dos, idesc, first);
          }
        }
      }
      mma_commit(empty0 + 8 * s);  // stage s free once these MMAs have read it
    }
    if (!ok) {
      atomicExch(abort_flag, 1);
      atomicOr(e.t.status, FQ_BIT_TIMEOUT);
    }
    mma_commit(done);  // arrives when every MMA issued above has completed
  }
  __syncwarp();

  // ---------------- epilogue: all 128 threads, thread = state row j, 16 columns at a time
  const bool got = mbar_wait(done, 0);
  tc_fence_after();
  if (!got) atomicOr(e.t.status, FQ_BIT_TIMEOUT);
  const bool run = got && !*(volatile int*)abort_flag;
  const int j = j0 + warp * 32 + lane;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  bool bad = false;
  double dsr = 0.0, dsi = 0.0;  // DOT partial of this thread
#pragma unroll 1
  for (int c0 = 0; c0 < BN; c0 += 16) {
    float yr[16], yi[16];
    tmem_ld16(trow + c0, yr);
    tmem_ld16(trow + BN + c0, yi);
    tmem_wait_ld();
    const int ib = i0 + c0;
    if (!run || j >= e.nc || ib >= e.n) continue;
    epi_chunk<NS, EPI>(e, yr, yi, j, ib, bad, dsr, dsi);
  }
  if (bad) atomicOr(e.t.status, FQ_BIT_BOUND);
  if (EPI == EPI_DOT) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dsr += __shfl_xor_sync(0xffffffffu, dsr, o);
      dsi += __shfl_xor_sync(0xffffffffu, dsi, o);
    }
    if (lane == 0) {
      red[2 * warp] = dsr;
      red[2 * warp + 1] = dsi;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (EPI == EPI_DOT && threadIdx.x == 0)
    e.partial[tj * tiles_i + ti] = make_double2(red[0] + red[2] + red[4] + red[6], red[1] + red[3] + red[5] + red[7]);
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)Cfg::TMEM_COLS)
                 : "memory");
  }
}

// Persistent form of k_split_term for the forward and adjoint epilogues: one CTA per SM walks
// the tiles blockIdx.x, blockIdx.x + gridDim.x, ...  Warp 0 (one thread) streams TMA stages,
// warp 1 (one thread) issues the MMAs of tile i into tensor-memory buffer i & 1, and warps 2-5
// run the epilogue of tile i from its buffer while tile i + 1 accumulates in the other one.
// Buffers are handed over by mbarriers (tfull: MMAs of a tile done; tempty: its accumulators
// read).  Every wait is bounded as in k_split_term.
constexpr int PTHREADS = 192;

template <int NS, int BN, int BKE, int EPI, bool HAS_A>
__global__ void __launch_bounds__(PTHREADS, 1)
k_split_persist(const __grid_constant__ SplitMaps maps, int nk, int tiles_j, int tiles_i, SplitEpi e) {
  static_assert(EPI != EPI_DOT, "the gradient dot keeps the one-tile kernel (per-CTA partials)");
  using Cfg = SplitCfg<NS, BN, BKE, HAS_A>;
  constexpr int STAGES = Cfg::STAGES;
  constexpr uint32_t BUF_COLS = 2 * BN;             // Yr and Yi of one tile
  constexpr uint32_t TMEM_COLS = 2 * BUF_COLS;      // two buffers (<= 512)
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = smem_raw + (base - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + STAGES * Cfg::STAGE_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 5);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES);
  const uint32_t tfull0 = smem_u32(bars + 2 * STAGES), tempty0 = smem_u32(bars + 2 * STAGES + 2);
  const uint32_t done = smem_u32(bars + 2 * STAGES + 4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = tiles_i * tiles_j;

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

  auto coords = [&](int t, int& j0, int& i0) {
    const int per = RASTER_GROUP * tiles_i, g = t / per;
    const int gj = min(RASTER_GROUP, tiles_j - g * RASTER_GROUP), r = t - g * per;
    j0 = (g * RASTER_GROUP + r % gj) * BM;
    i0 = (r / gj) * BN;
  };

  if (warp == 0) {
    if (lane == 0) {  // ---------------- TMA producer
      int g = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        int j0, i0;
        coords(t, j0, i0);
        for (int kb = 0; kb < nk; ++kb) {
          const int s = g % STAGES;
          if (g >= STAGES && !(ok = mbar_wait(empty0 + 8 * s, ((g / STAGES) - 1) & 1))) break;
          if (*(volatile int*)abort_flag) {
            ok = false;
            break;
          }
          const uint32_t st = base + s * Cfg::STAGE_BYTES;
          const uint32_t bar = full0 + 8 * s;
          mbar_expect_tx(bar, Cfg::STAGE_BYTES);
          const int kx = kb * BKE;
#pragma unroll
          for (int q = 0; q < NS; ++q) {
            tma_load_2d(st + q * Cfg::A_BYTES, &maps.a[q], bar, kx, j0);
            tma_load_2d(st + (NS + q) * Cfg::A_BYTES, &maps.a[q], bar, e.np + kx, j0);
            tma_load_2d(st + 2 * NS * Cfg::A_BYTES + q * Cfg::B_BYTES, &maps.os[q], bar, kx, i0);
            if (HAS_A)
              tma_load_2d(st + 2 * NS * Cfg::A_BYTES + (NS + q) * Cfg::B_BYTES, &maps.oa[q], bar, kx, i0);
          }
          ++g;
        }
      }
      if (!ok) {
        atomicExch(abort_flag, 1);
        atomicOr(e.t.status, FQ_BIT_TIMEOUT);
      }
      // every copy issued must have landed before the CTA may exit
      for (int q = max(0, g - STAGES); q < g; ++q) mbar_wait(full0 + 8 * (q % STAGES), (q / STAGES) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ---------------- MMA issuer
      constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                 ((uint32_t)(BM >> 4) << 24);
      constexpr uint32_t idesc_neg = idesc | (1u << 13);
      int g = 0, i = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++i) {
        const int b = i & 1;
        if (i >= 2 && !(ok = mbar_wait(tempty0 + 8 * b, ((i >> 1) - 1) & 1))) break;
        const uint32_t acc = tmem + (uint32_t)b * BUF_COLS;
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = g % STAGES;
          ok = mbar_wait(full0 + 8 * s, (g / STAGES) & 1);
          if (!ok || *(volatile int*)abort_flag) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = base + s * Cfg::STAGE_BYTES;
#pragma unroll
          for (int p = 0; p < Pairs<NS>::N; ++p) {
            const uint32_t pr = st + Pairs<NS>::a(p) * Cfg::A_BYTES;
            const uint32_t pi = st + (NS + Pairs<NS>::a(p)) * Cfg::A_BYTES;
            const uint32_t os = st + 2 * NS * Cfg::A_BYTES + Pairs<NS>::b(p) * Cfg::B_BYTES;
            const uint32_t oa = st + 2 * NS * Cfg::A_BYTES + (NS + Pairs<NS>::b(p)) * Cfg::B_BYTES;
#pragma unroll
            for (int kk = 0; kk < BKE / 16; ++kk) {
              const uint32_t first = (kb == 0 && p == 0 && kk == 0) ? 0u : 1u;
              const uint64_t dpr = smem_desc<Cfg::ROWB>(pr + 32 * kk), dpi = smem_desc<Cfg::ROWB>(pi + 32 * kk);
              const uint64_t dos = smem_desc<Cfg::ROWB>(os + 32 * kk);
              if (HAS_A) {
                const uint64_t doa = smem_desc<Cfg::ROWB>(oa + 32 * kk);
                mma_bf16(acc, dpr, dos, idesc, first);
                mma_bf16(acc, dpi, doa, idesc_neg, 1u);
                mma_bf16(acc + BN, dpr, doa, idesc, first);
                mma_bf16(acc + BN, dpi, dos, idesc, 1u);
              } else {
                mma_bf16(acc, dpr, dos, idesc, first);
                mma_bf16(acc + BN, dpi, dos, idesc, first);
              }
            }
          }
          mma_commit(empty0 + 8 * s);
        }
        if (!ok) break;
        mma_commit(tfull0 + 8 * b);  // this tile's accumulators are complete once its MMAs are
      }
      if (!ok) {
        atomicExch(abort_flag, 1);
        atomicOr(e.t.status, FQ_BIT_TIMEOUT);
      }
      mma_commit(done);  // every MMA issued above has completed once this arrives
      mbar_wait(done, 0);
    }
  } else {  // ---------------- epilogue warps 2-5: tensor-memory lane quarter warp % 4
    const int quarter = warp & 3;
    bool bad = false, ok = true;
    double dsr = 0.0, dsi = 0.0;
    int i = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      const int b = i & 1;
      bool go = mbar_wait(tfull0 + 8 * b, (i >> 1) & 1);
      tc_fence_after();
      go = __all_sync(0xffffffffu, go && !*(volatile int*)abort_flag);  // warp-uniform: tcgen05.ld is .aligned
      if (!go) {
        ok = false;
        break;
      }
      int j0, i0;
      coords(t, j0, i0);
      const int j = j0 + quarter * 32 + lane;
      const uint32_t trow = tmem + (uint32_t)b * BUF_COLS + ((uint32_t)(quarter * 32) << 16);
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 16) {
        float yr[16], yi[16];
        tmem_ld16(trow + c0, yr);
        tmem_ld16(trow + BN + c0, yi);
        tmem_wait_ld();
        const int ib = i0 + c0;
        if (j >= e.nc || ib >= e.n) continue;
        epi_chunk<NS, EPI>(e, yr, yi, j, ib, bad, dsr, dsi);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty0 + 8 * b);
    }
    if (!ok) {
      atomicExch(abort_flag, 1);
      atomicOr(e.t.status, FQ_BIT_TIMEOUT);
    }
    if (bad) atomicOr(e.t.status, FQ_BIT_BOUND);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// ------------------------------------------------------------------------- chained products
// A chain of dependent products Y_p = left_p . right^T, p = 0 .. nprod-1, with one right operand
// (a step's Omega~_m) and product p's left operand written by product p-1's epilogue: the L
// Chebyshev terms of a step (forward or adjoint).  One cooperative launch runs the whole chain:
// work unit u = p * tiles + t (tiles in row-block-major order), CTA c takes the units c, c + G, ...
// in increasing order.  Product p's tiles of state-row block tj need exactly the rows tj of its left
// operand, i.e. the epilogues of product p-1's tiles (tj, *): a counter per (p - 1, tj) counts their
// epilogue warps, and the TMA producer waits for it (bounded) before loading.  A unit waits only on units with a
// smaller index, and all CTAs are resident (cooperative launch), so the chain always advances; the
// epilogue of one unit overlaps the MMAs of the next as in k_split_persist.
constexpr int CHAIN_MAXP = 12;

struct ChainArgs {
  SplitMaps rmaps;                 // right operand (os, oa); its a[] is unused
  CUtensorMap left[CHAIN_MAXP][3]; // left operand slices of product p
  SplitEpi epi[CHAIN_MAXP];        // epilogue of product p (slice_out = product p+1's left operand)
  int nprod, nk, tiles_j, tiles_i;
  unsigned int* flags;             // [nprod][tiles_j]: finished epilogue warps (4 a tile) of product p in
                                   // row block tj (zeroed before the launch)
};

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
// bounded wait until *p >= target (acquire); false if it gave up
__device__ __forceinline__ bool wait_count(const unsigned int* p, unsigned int target) {
  const long long t0 = clock64();
  while (ld_acquire_u32(p) < target) {
    if (clock64() - t0 > kWaitCycles) return false;
    __nanosleep(64);
  }
  return true;
}

template <int NS, int BN, int BKE, int EPI, bool HAS_A>
__global__ void __launch_bounds__(PTHREADS, 1) k_split_chain(const __grid_constant__ ChainArgs args) {
  static_assert(EPI != EPI_DOT, "chains of forward or adjoint terms only");
  using Cfg = SplitCfg<NS, BN, BKE, HAS_A>;
  constexpr int STAGES = Cfg::STAGES;
  constexpr uint32_t BUF_COLS = 2 * BN;
  constexpr uint32_t TMEM_COLS = 2 * BUF_COLS;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = smem_raw + (base - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + STAGES * Cfg::STAGE_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 5);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES);
  const uint32_t tfull0 = smem_u32(bars + 2 * STAGES), tempty0 = smem_u32(bars + 2 * STAGES + 2);
  const uint32_t done = smem_u32(bars + 2 * STAGES + 4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles = args.tiles_i * args.tiles_j;
  const int nunits = args.nprod * tiles;
  unsigned int* status = args.epi[0].t.status;

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

  auto unit = [&](int u, int& p, int& tj, int& j0, int& i0) {
    p = u / tiles;
    const int t = u - p * tiles;
    tj = t / args.tiles_i;
    j0 = tj * BM;
    i0 = (t - tj * args.tiles_i) * BN;
  };

  if (warp == 0) {
    if (lane == 0) {  // ---------------- TMA producer: waits for each unit's left operand
      int g = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        int p, tj, j0, i0;
        unit(u, p, tj, j0, i0);
        if (p > 0) {
          if (!(ok = wait_count(args.flags + (size_t)(p - 1) * args.tiles_j + tj, 4u * args.tiles_i))) break;
          fence_proxy_async_global();  // the epilogues' generic stores, before this thread's TMA reads
        }
        const int np_ = args.epi[p].np;
        for (int kb = 0; kb < args.nk; ++kb) {
          const int s = g % STAGES;
          if (g >= STAGES && !(ok = mbar_wait(empty0 + 8 * s, ((g / STAGES) - 1) & 1))) break;
          if (*(volatile int*)abort_flag) {
            ok = false;
            break;
          }
          const uint32_t st = base + s * Cfg::STAGE_BYTES;
          const uint32_t bar = full0 + 8 * s;
          mbar_expect_tx(bar, Cfg::STAGE_BYTES);
          const int kx = kb * BKE;
#pragma unroll
          for (int q = 0; q < NS; ++q) {
            tma_load_2d(st + q * Cfg::A_BYTES, &args.left[p][q], bar, kx, j0);
            tma_load_2d(st + (NS + q) * Cfg::A_BYTES, &args.left[p][q], bar, np_ + kx, j0);
            tma_load_2d(st + 2 * NS * Cfg::A_BYTES + q * Cfg::B_BYTES, &args.rmaps.os[q], bar, kx, i0);
            if (HAS_A)
              tma_load_2d(st + 2 * NS * Cfg::A_BYTES + (NS + q) * Cfg::B_BYTES, &args.rmaps.oa[q], bar, kx, i0);
          }
          ++g;
        }
      }
      if (!ok) {
        atomicExch(abort_flag, 1);
        atomicOr(status, FQ_BIT_TIMEOUT);
      }
      for (int q = max(0, g - STAGES); q < g; ++q) mbar_wait(full0 + 8 * (q % STAGES), (q / STAGES) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ---------------- MMA issuer (as k_split_persist)
      constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                 ((uint32_t)(BM >> 4) << 24);
      constexpr uint32_t idesc_neg = idesc | (1u << 13);
      int g = 0, i = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x, ++i) {
        const int b = i & 1;
        if (i >= 2 && !(ok = mbar_wait(tempty0 + 8 * b, ((i >> 1) - 1) & 1))) break;
        const uint32_t acc = tmem + (uint32_t)b * BUF_COLS;
        for (int kb = 0; kb < args.nk; ++kb, ++g) {
          const int s = g % STAGES;
          ok = mbar_wait(full0 + 8 * s, (g / STAGES) & 1);
          if (!ok || *(volatile int*)abort_flag) {
            ok = false;
            break;
          }
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
              const uint64_t dos = smem_desc<Cfg::ROWB>(os + 32 * kk);
              if (HAS_A) {
                const uint64_t doa = smem_desc<Cfg::ROWB>(oa + 32 * kk);
                mma_bf16(acc, dpr, dos, idesc, first);
                mma_bf16(acc, dpi, doa, idesc_neg, 1u);
                mma_bf16(acc + BN, dpr, doa, idesc, first);
                mma_bf16(acc + BN, dpi, dos, idesc, 1u);
              } else {
                mma_bf16(acc, dpr, dos, idesc, first);
                mma_bf16(acc + BN, dpi, dos, idesc, first);
              }
            }
          }
          mma_commit(empty0 + 8 * s);
        }
        if (!ok) break;
        mma_commit(tfull0 + 8 * b);
      }
      if (!ok) {
        atomicExch(abort_flag, 1);
        atomicOr(status, FQ_BIT_TIMEOUT);
      }
      mma_commit(done);
      mbar_wait(done, 0);
    }
  } else {  // ---------------- epilogue warps 2-5; then the unit's completion for its row block
    const int quarter = warp & 3;
    bool bad = false, ok = true;
    double dsr = 0.0, dsi = 0.0;
    int i = 0;
    for (int u = blockIdx.x; u < nunits; u += gridDim.x, ++i) {
      int p, tj, j0, i0;
      unit(u, p, tj, j0, i0);
      const int b = i & 1;
      bool go = mbar_wait(tfull0 + 8 * b, (i >> 1) & 1);
      tc_fence_after();
      go = __all_sync(0xffffffffu, go && !*(volatile int*)abort_flag);
      if (!go) {
        ok = false;
        break;
      }
      // the previous product's outputs this epilogue reads (prev, acc) were released with its counter
      if (p > 0) ld_acquire_u32(args.flags + (size_t)(p - 1) * args.tiles_j + tj);
      const SplitEpi& e = args.epi[p];
      const int j = j0 + quarter * 32 + lane;
      const uint32_t trow = tmem + (uint32_t)b * BUF_COLS + ((uint32_t)(quarter * 32) << 16);
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 16) {
        float yr[16], yi[16];
        tmem_ld16(trow + c0, yr);
        tmem_ld16(trow + BN + c0, yi);
        tmem_wait_ld();
        const int ib = i0 + c0;
        if (j >= e.nc || ib >= e.n) continue;
        epi_chunk<NS, EPI>(e, yr, yi, j, ib, bad, dsr, dsi);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty0 + 8 * b);
      // this warp's stores of the unit made visible (to the async proxy too), then one release per
      // warp: a tile is done when its four epilogue warps have counted
      fence_proxy_async_global();
      __threadfence();
      __syncwarp();
      if (lane == 0) red_release_add(args.flags + (size_t)p * args.tiles_j + tj, 1u);
    }
    if (!ok) {
      atomicExch(abort_flag, 1);
      atomicOr(status, FQ_BIT_TIMEOUT);
    }
    if (bad) atomicOr(status, FQ_BIT_BOUND);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// Launches a chain cooperatively (all CTAs resident).  FQ_EUNSUPPORTED when that cannot be done
// (a capturing stream, or the device refuses the cooperative launch): the caller then runs the
// products one launch each.
template <int NS, int BN, int BKE, int EPI, bool HAS_A>
fq_status launch_chain(const ChainArgs& args, cudaStream_t s) {
  using Cfg = SplitCfg<NS, BN, BKE, HAS_A>;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return FQ_EUNSUPPORTED;
  static std::atomic<unsigned> attr_set{0};
  if (fq_first_on_device(attr_set)) {
    cudaError_t e = cudaFuncSetAttribute(k_split_chain<NS, BN, BKE, EPI, HAS_A>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
    if (e != cudaSuccess) return fq_cuda_fail(e, "chain kernel shared-memory attribute");
  }
  const int tiles = args.tiles_i * args.tiles_j;
  const int grid = std::min(tiles, fq_sm_count());
  void* kargs[] = {(void*)&args};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_split_chain<NS, BN, BKE, EPI, HAS_A>, dim3(grid),
                                              dim3(PTHREADS), kargs, Cfg::SMEM, s);
  if (e == cudaErrorCooperativeLaunchTooLarge || e == cudaErrorNotSupported) {
    cudaGetLastError();
    return FQ_EUNSUPPORTED;
  }
  return e == cudaSuccess ? FQ_OK : fq_cuda_fail(e, "chain kernel launch");
}

// ------------------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

fq_status encode_fn() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  });
  if (!g_encode) {
    fq_set_error("cuTensorMapEncodeTiled is not available from the driver");
    return FQ_ECUDA;
  }
  return FQ_OK;
}

// 2-D BF16 map over [rows][cols] (row-major, cols contiguous), box = box_cols x box_rows with the
// swizzle matching box_cols * 2 bytes (128, 64 or 32).
fq_status make_map(CUtensorMap* m, const void* ptr, int rows, int cols, int box_rows, int box_cols) {
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapSwizzle sw = box_cols == 64   ? CU_TENSOR_MAP_SWIZZLE_128B
                                : box_cols == 32 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                 : CU_TENSOR_MAP_SWIZZLE_32B;
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    fq_set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return FQ_ECUDA;
  }
  return FQ_OK;
}

int grid_1d(size_t total) { return (int)std::min<size_t>(std::max<size_t>((total + 255) / 256, 1), 152 * 32); }

}  // namespace
