// Split-precision dense Chebyshev term on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// One term of Eq. 10 on a block of nc state rows: Y^T = Psi^T Omega~^T with Omega~ = S + i A
// (S real symmetric, A real antisymmetric), i.e. with X.B := sum_k X[j][k] B[i][k]
//   Yr = Psi_r.S - Psi_i.A,   Yi = Psi_r.A + Psi_i.S.
// Each K stage loads the Psi_r, Psi_i tiles and one S and one A tile, and four MMA streams
// (the minus sign through the instruction's negate-A bit) use every tile twice.  Every operand
// is held as NS BF16 slices
// (x = x_0 + x_1 + ..., x_s = bf16 of the remainder), and the products x_a y_b with a + b < NS
// (3 for NS = 2, 6 for NS = 3) are summed in FP32 in tensor memory.  The epilogue applies the
// recurrence psi_{l+1} = -2i Y + psi_{l-1}, the Bessel accumulation and the step phase on FP32
// master copies (Eqs. 10, 12) and writes the next term's slices.
//
// CTA: 128 threads, tile 128 state rows x BN output columns, tiles rasterized in groups of 8 row
// blocks so that co-running CTAs share operands in L2.  Thread 0 of warp 0 issues TMA loads
// (K-major, 128- or 64-byte swizzle), thread 0 of warp 1 issues tcgen05.mma (A and B from shared memory,
// D in tensor memory), stages handed over by mbarriers; all four warps read the accumulators
// back with tcgen05.ld for the epilogue.  Every wait is bounded; a wait that gives up records
// FQ_BIT_TIMEOUT, drains this CTA's own copies and MMAs, frees tensor memory and returns.
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

struct SplitMaps {
  CUtensorMap a[3];   // left operand slices [ncp][2 Np]: Psi_r in columns [0, Np), Psi_i in [Np, 2 Np)
  CUtensorMap os[3];  // S slices [Np][Np]
  CUtensorMap oa[3];  // A slices [Np][Np]
};

struct SplitEpi {
  int n, nc, ldm, np;          // dims; ldm: FP32 master row stride; np: real part width in K'
  const float* cur_re;         // psi_l masters (first term: psi_0)
  const float* cur_im;
  const float* prev_re;        // psi_{l-1}
  const float* prev_im;
  float* acc_re;
  float* acc_im;
  float* out_re;               // psi_{l+1} (in place of psi_{l-1}) or X at the last term
  float* out_im;
  __nv_bfloat16* slice_out;    // next left operand: NS slices, each [nc][Kp]
  size_t slice_stride;         // elements between slices
  int kp;
  fq_term t;
};

template <int NS, int BN, int BKE>
struct SplitCfg {
  static constexpr int ROWB = BKE * 2;                // bytes per K row of a stage (swizzle span)
  static constexpr int A_BYTES = BM * ROWB;           // one slice of Psi_r or Psi_i, one stage
  static constexpr int B_BYTES = BN * ROWB;           // one slice of S or A, one stage
  static constexpr int STAGE_BYTES = 2 * NS * A_BYTES + 2 * NS * B_BYTES;
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

template <int NS, int BN, int BKE>
__global__ void __launch_bounds__(NTHREADS, 1)
k_split_term(const __grid_constant__ SplitMaps maps, int nk, int tiles_j, int tiles_i, SplitEpi e) {
  using Cfg = SplitCfg<NS, BN, BKE>;
  constexpr int STAGES = Cfg::STAGES;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned stage buffers (swizzle atoms), then barriers
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = smem_raw + (base - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + STAGES * Cfg::STAGE_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
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
        tma_load_2d(st + 2 * NS * Cfg::A_BYTES + q * Cfg::B_BYTES, &maps.os[q], bar, kx, i0);         // S
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
    // ---------------- MMA issuer: Yr += Psi_r.S - Psi_i.A, Yi += Psi_r.A + Psi_i.S
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
          const uint64_t dos = smem_desc<Cfg::ROWB>(os + 32 * kk), doa = smem_desc<Cfg::ROWB>(oa + 32 * kk);
          mma_bf16(tmem, dpr, dos, idesc, first);
          mma_bf16(tmem, dpi, doa, idesc_neg, 1u);
          mma_bf16(tmem + BN, dpr, doa, idesc, first);
          mma_bf16(tmem + BN, dpi, dos, idesc, 1u);
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
  const float c0f = (float)e.t.coef0, cf = (float)e.t.coef, pr_ = (float)e.t.ph_re, pi_ = (float)e.t.ph_im;
  const float b2 = (float)e.t.bound2;
  bool bad = false;
#pragma unroll 1
  for (int c0 = 0; c0 < BN; c0 += 16) {
    float yr[16], yi[16];
    tmem_ld16(trow + c0, yr);
    tmem_ld16(trow + BN + c0, yi);
    tmem_wait_ld();
    const int ib = i0 + c0;
    if (!run || j >= e.nc || ib >= e.n) continue;
    const int cnt = min(16, e.n - ib);
    const size_t idx = (size_t)j * e.ldm + ib;
    float a_r[16], a_i[16], p_r[16], p_i[16];
    const float* src_r = e.t.first ? e.cur_re : e.prev_re;
    const float* src_i = e.t.first ? e.cur_im : e.prev_im;
    if (cnt == 16) {
#pragma unroll
      for (int q = 0; q < 16; q += 4) {
        load_f4(src_r + idx + q, p_r + q);
        load_f4(src_i + idx + q, p_i + q);
        if (!e.t.first) {
          load_f4(e.acc_re + idx + q, a_r + q);
          load_f4(e.acc_im + idx + q, a_i + q);
        }
      }
    } else {
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const bool in = q < cnt;
        p_r[q] = in ? src_r[idx + q] : 0.f;
        p_i[q] = in ? src_i[idx + q] : 0.f;
        a_r[q] = (in && !e.t.first) ? e.acc_re[idx + q] : 0.f;
        a_i[q] = (in && !e.t.first) ? e.acc_im[idx + q] : 0.f;
      }
    }
    float o_r[16], o_i[16];
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
    // slices of the 16 new entries, packed two bf16 per 32-bit word (element 2w in the low half)
    uint32_t wre[NS][8], wim[NS][8];
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
      for (int q = 0; q < 16; q += 4) {
        store_f4(e.out_re + idx + q, o_r + q);
        store_f4(e.out_im + idx + q, o_i + q);
        if (!e.t.last) {
          store_f4(e.acc_re + idx + q, a_r + q);
          store_f4(e.acc_im + idx + q, a_i + q);
        }
      }
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
          e.out_re[idx + q] = o_r[q];
          e.out_im[idx + q] = o_i[q];
          if (!e.t.last) {
            e.acc_re[idx + q] = a_r[q];
            e.acc_im[idx + q] = a_i[q];
          }
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
  if (bad) atomicOr(e.t.status, FQ_BIT_BOUND);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)Cfg::TMEM_COLS)
                 : "memory");
  }
}

// Right operands of step m: S and A of Omega~_m = S + i A as NS BF16 slices [Np][Np] each, computed
// in FP64 (stage a2): S = sa H0 + sb H1 - sbeta 1, A = sc [H0,H1]; zero outside N x N.
template <int NS>
__global__ void k_split_omega(const double* __restrict__ h0, const double* __restrict__ h1,
                              const double* __restrict__ k, int n, int np, double sa, double sb, double sc,
                              double sbeta, __nv_bfloat16* os, __nv_bfloat16* oa, size_t slice_stride) {
  const size_t total = (size_t)np * np;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(q / np), c = (int)(q % np);
    double S = 0.0, A = 0.0;
    if (i < n && c < n) {
      const size_t o = (size_t)i * n + c;
      S = sa * h0[o] + sb * h1[o] - (i == c ? sbeta : 0.0);
      A = sc * k[o];
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
// swizzle matching box_cols * 2 bytes (128 or 64).
fq_status make_map(CUtensorMap* m, const void* ptr, int rows, int cols, int box_rows, int box_cols) {
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapSwizzle sw = box_cols == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
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

// ------------------------------------------------------------------------- orchestration
// Workspace: B slices (Br, Bi), two left-operand slice buffers (ping-pong across terms), three
// FP32 master state buffers (planar) for psi_l / psi_{l-1} / acc.
struct SplitWs {
  __nv_bfloat16* os;  // S slices
  __nv_bfloat16* oa;  // A slices
  __nv_bfloat16* a[2];
  float* m[3][2];
  int np, kp, ldm, ncp;
  size_t bstride, astride;
};

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
  if (out) *(SplitWs*)out = w;
  return off;
}

template <int NS, int BN, int BKE>
static fq_status run_split(fq_plan* p, const double* x0, double* x, int nc, int m_begin, int m_end, int identity,
                           int transpose_out, void* ws, cudaStream_t s) {
  using Cfg = SplitCfg<NS, BN, BKE>;
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
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_split_term<NS, BN, BKE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Cfg::SMEM);
    if (e != cudaSuccess) return fq_cuda_fail(e, "split kernel smem attribute");
    attr = true;
  }
  // left-operand slices are only ever written for rows < nc and columns < n: zero the padding
  cudaMemsetAsync(w.a[0], 0, sizeof(__nv_bfloat16) * NS * w.astride, s);
  cudaMemsetAsync(w.a[1], 0, sizeof(__nv_bfloat16) * NS * w.astride, s);
  k_split_init<NS><<<grid_1d((size_t)nc * w.kp), 256, 0, s>>>(identity ? nullptr : (const double2*)x0, n, nc, w.ldm,
                                                               w.np, w.kp, w.m[0][0], w.m[0][1], w.a[0], w.astride);
  const int tiles_i = w.np / BN, tiles_j = (nc + BM - 1) / BM;
  const dim3 grid(tiles_i * tiles_j);
  const int nk = w.np / BKE;
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
      k_split_omega<NS><<<grid_1d(w.bstride), 256, 0, s>>>(p->d_h0, p->d_h1, p->d_k, n, w.np, p->sa[m], p->sb[m],
                                                           p->sc[m], p->sbeta, w.os, w.oa, w.bstride);
    }
    int cur = xb, nxt = (xb + 1) % 3, acc = (xb + 2) % 3, prv = -1;
    for (int l = 0; l < L; ++l) {
      t.first = l == 0;
      t.last = l == L - 1;
      t.coef = p->cheb[l + 1];
      const int out = l == 0 ? nxt : prv;
      SplitEpi e{};
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
      k_split_term<NS, BN, BKE><<<grid, NTHREADS, Cfg::SMEM, s>>>(maps[av], nk, tiles_j, tiles_i, e);
      av ^= 1;
      if (t.last) {
        xb = out;
      } else {
        prv = cur;
        cur = out;
      }
    }
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
  return wide ? run_split<2, 128, 32>(p, x0, x, nc, m_begin, m_end, identity, transpose_out, ws, s)
              : run_split<2, 64, 64>(p, x0, x, nc, m_begin, m_end, identity, transpose_out, ws, s);
}

// Times each tile width on two steps of the identity block and keeps the fastest.
extern "C" fq_status floquet_autotune(fq_plan* p, void* ws, size_t bytes, void* stream, int32_t* tile_n) {
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
  const int cand[2] = {64, 128};
  float best = 1e30f;
  int pick = 64;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  for (int c : cand) {
    p->tile_n = c;
    fq_status st = fq_split_propagate(p, nullptr, nullptr, p->n, 0, steps, 1, 0, ws, s);  // warm-up
    if (st != FQ_OK) break;
    cudaEventRecord(a, s);
    fq_split_propagate(p, nullptr, nullptr, p->n, 0, steps, 1, 0, ws, s);
    cudaEventRecord(b, s);
    cudaError_t e = cudaEventSynchronize(b);
    if (e != cudaSuccess) {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      return fq_cuda_fail(e, "autotune");
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (ms < best) {
      best = ms;
      pick = c;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  p->tile_n = pick;
  if (tile_n) *tile_n = pick;
  return FQ_OK;
}
