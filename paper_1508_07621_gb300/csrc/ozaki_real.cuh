// FP64 emulation of the products with a real right operand (the gradient's forward, adjoint and
// dot products: Omega~_m and E = H1 / Delta E are real symmetric there), with stacked rows.
//
// The real and imaginary parts of 64 states are stacked as the 128 rows of the MMA's left
// operand (rows 0-63: Re psi, rows 64-127: Im psi), so one MMA of N = 64 per slice pair makes both
// Y_r and Y_i of a 64 x 64 tile, and one accumulator group takes 64 tensor-memory columns.  The
// four groups of ozaki_core.cuh (three exact ones and the tail) then fill half of the tensor
// memory, and the chunks of K alternate between two halves: the drain warps fold chunk c while
// the MMAs of chunk c + 1 run.  With one MMA per pair and value of k, a group's sum over 256
// values of k is at most 3 pairs x 2^14 x 256 < 2^24 units: still exact.
//
// Warp 0 streams TMA stages (K = 16 per stage: the two 64-row halves of each left slice and the
// 64 rows of each right slice), warp 1 issues the MMAs, warps 2-17 drain (four per lane quarter,
// 16 columns each) and finally run the FP64 epilogue on 8 columns of one state each.  Every wait
// is bounded as in the other tensor-core kernels.
#pragma once

#include "ozaki_core.cuh"

namespace {

constexpr int OZR_BM = 64;                        // states per tile (128 stacked rows)
constexpr int OZR_A_BYTES = 2 * OZR_BM * OZ_ROWB; // one left slice: Re and Im halves, 4 KB
constexpr int OZR_B_BYTES = OZ_BN * OZ_ROWB;      // one right slice, 2 KB
constexpr int OZR_STAGE_BYTES = OZ_S * (OZR_A_BYTES + OZR_B_BYTES);
constexpr int OZR_STAGES = 4;
constexpr int OZR_KB_PER_DRAIN = 16;              // 256 values of k per chunk
constexpr int OZR_BUF_COLS = 4 * OZ_BN;           // four groups of 64 columns
constexpr int OZR_XS_LD = 129;                    // staged sums: [col][row], padded against bank conflicts
constexpr int OZR_XS_BYTES = 2 * OZR_XS_LD * OZ_BN * 4;  // hi, then lo
constexpr size_t OZR_SMEM = (size_t)OZR_STAGES * OZR_STAGE_BYTES + 1024 + 256;
static_assert((size_t)OZR_STAGES * OZR_STAGE_BYTES >= OZR_XS_BYTES + 16 * sizeof(double2), "epilogue staging");

template <int EPI>
__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_oz_real_term(const __grid_constant__ OzMaps maps, int nk, int tiles_j, int tiles_i, int np, OzEpi e) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = smem_raw + (base - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + OZR_STAGES * OZR_STAGE_BYTES);
  // full[4], empty[4], tfull[2], tempty[2], done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * OZR_STAGES + 5);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + OZR_STAGES);
  const uint32_t tfull0 = smem_u32(bars + 2 * OZR_STAGES), tempty0 = smem_u32(bars + 2 * OZR_STAGES + 2);
  const uint32_t done = smem_u32(bars + 2 * OZR_STAGES + 4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchunks = (nk + OZR_KB_PER_DRAIN - 1) / OZR_KB_PER_DRAIN;

  int tj, ti;
  {
    const int b = blockIdx.x, per = RASTER_GROUP * tiles_i, g = b / per;
    const int gj = min(RASTER_GROUP, tiles_j - g * RASTER_GROUP), r = b - g * per;
    tj = g * RASTER_GROUP + r % gj;
    ti = r / gj;
  }
  const int j0 = tj * OZR_BM, i0 = ti * OZ_BN;

  if (threadIdx.x == 0) {
    for (int s = 0; s < OZR_STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull0 + 8 * b, 1);
      mbar_init(tempty0 + 8 * b, OZ_EPI_WARPS);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(OZ_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {  // ---------------- TMA producer
      int issued = 0;
      bool ok = true;
      for (int kb = 0; kb < nk && ok; ++kb) {
        const int s = kb % OZR_STAGES;
        if (kb >= OZR_STAGES && !(ok = mbar_wait(empty0 + 8 * s, ((kb / OZR_STAGES) - 1) & 1))) break;
        if (*(volatile int*)abort_flag) {
          ok = false;
          break;
        }
        const uint32_t st = base + s * OZR_STAGE_BYTES;
        const uint32_t bar = full0 + 8 * s;
        mbar_expect_tx(bar, OZR_STAGE_BYTES);
        const int kx = kb * OZ_BKE;
#pragma unroll
        for (int q = 0; q < OZ_S; ++q) {
          tma_load_2d(st + q * OZR_A_BYTES, &maps.a[q], bar, kx, j0);                                // Re rows
          tma_load_2d(st + q * OZR_A_BYTES + OZR_BM * OZ_ROWB, &maps.a[q], bar, np + kx, j0);        // Im rows
          tma_load_2d(st + OZ_S * OZR_A_BYTES + q * OZR_B_BYTES, &maps.r[q], bar, kx, i0);           // S rows
        }
        issued = kb + 1;
      }
      if (!ok) {
        atomicExch(abort_flag, 1);
        atomicOr(e.t.status, FQ_BIT_TIMEOUT);
      }
      for (int kb = max(0, issued - OZR_STAGES); kb < issued; ++kb)
        mbar_wait(full0 + 8 * (kb % OZR_STAGES), (kb / OZR_STAGES) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ---------------- MMA issuer
      constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OZ_BN >> 3) << 17) |
                                 ((uint32_t)(128 >> 4) << 24);
      bool ok = true;
      int kb = 0;
      for (int c = 0; c < nchunks && ok; ++c) {
        const int b = c & 1;
        if (c >= 2 && !(ok = mbar_wait(tempty0 + 8 * b, ((c >> 1) - 1) & 1))) break;
        tc_fence_after();
        const uint32_t accb = tmem + (uint32_t)(b * OZR_BUF_COLS);
        for (int kq = 0; kq < OZR_KB_PER_DRAIN && kb < nk; ++kq, ++kb) {
          const int s = kb % OZR_STAGES;
          ok = mbar_wait(full0 + 8 * s, (kb / OZR_STAGES) & 1);
          if (!ok || *(volatile int*)abort_flag) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t d0 = oz_desc(base + s * OZR_STAGE_BYTES);
#pragma unroll
          for (int p = 0; p < OZ_PAIRS; ++p) {
            int a, bb;
            oz_pair(p, a, bb);
            const int g = a + bb < 3 ? a + bb : 3;
            const bool lead = p == 0 || p == 1 || p == 3 || p == 6;
            mma_bf16(accb + (uint32_t)(g * OZ_BN), d0 + (uint64_t)((a * OZR_A_BYTES) >> 4),
                     d0 + (uint64_t)((OZ_S * OZR_A_BYTES + bb * OZR_B_BYTES) >> 4), idesc,
                     (kq == 0 && lead) ? 0u : 1u);
          }
          mma_commit(empty0 + 8 * s);
        }
        if (!ok) break;
        mma_commit(tfull0 + 8 * b);
      }
      if (!ok) {
        atomicExch(abort_flag, 1);
        atomicOr(e.t.status, FQ_BIT_TIMEOUT);
      }
      mma_commit(done);
      mbar_wait(done, 0);
    }
  } else {  // ---------------- drain warps 2-17
    const int quarter = warp & 3, part = (warp - 2) >> 2;
    const int row = quarter * 32 + lane;  // stacked row: Re of state row (< 64), Im of state row - 64
    float2 h[8], l[8];                    // double-float sums of columns (2p, 2p + 1)
#pragma unroll
    for (int q = 0; q < 8; ++q) h[q] = l[q] = make_float2(0.f, 0.f);
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      const int b = c & 1;
      bool go = mbar_wait(tfull0 + 8 * b, (c >> 1) & 1);
      tc_fence_after();
      go = __all_sync(0xffffffffu, go && !*(volatile int*)abort_flag);
      if (!go) {
        ok = false;
        break;
      }
      const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * OZR_BUF_COLS + part * 16);
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        float v[16];
        tmem_ld16(trow + g * OZ_BN, v);
        tmem_wait_ld();
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float2 w = make_float2(v[2 * q], v[2 * q + 1]);
          if (g < 3) dd_add2(h[q], l[q], w);
          else l[q] = __fadd2_rn(l[q], w);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty0 + 8 * b);
    }
    if (!ok) {
      atomicExch(abort_flag, 1);
      atomicOr(e.t.status, FQ_BIT_TIMEOUT);
    }
    // stage the sums column-major (xs[col][row], hi then lo) in the idle stages: the last MMAs
    // have completed, and every stage's copies have landed
    float* xs = reinterpret_cast<float*>(gbase);
    constexpr int LO = OZR_XS_LD * OZ_BN;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int c0 = part * 16 + 2 * q;
      xs[c0 * OZR_XS_LD + row] = h[q].x;
      xs[(c0 + 1) * OZR_XS_LD + row] = h[q].y;
      xs[LO + c0 * OZR_XS_LD + row] = l[q].x;
      xs[LO + (c0 + 1) * OZR_XS_LD + row] = l[q].y;
    }
    asm volatile("bar.sync 1, %0;" ::"n"(32 * OZ_EPI_WARPS) : "memory");  // the drain warps only
    // ---------------- FP64 epilogue: thread t -> state t / 8, columns 8 (t % 8) .. + 7
    const int t = threadIdx.x - 64, srow = t >> 3, cb = (t & 7) * 8;
    const int j = j0 + srow;
    double dsr = 0.0, dsi = 0.0;
    bool bad = false;
    if (ok && j < e.nc) {
      const fq_term& tt = e.t;
      const int ej = e.es[j];
#pragma unroll 1
      for (int q = 0; q < 8; ++q) {
        const int cc = cb + q, i = i0 + cc;
        if (i >= e.n) break;
        const int ex = ej + e.et[i];
        const double sc = pow2(ex < -1022 ? -1022 : ex);
        const double yr = ((double)xs[cc * OZR_XS_LD + srow] + (double)xs[LO + cc * OZR_XS_LD + srow]) * sc;
        const double yi =
            ((double)xs[cc * OZR_XS_LD + 64 + srow] + (double)xs[LO + cc * OZR_XS_LD + 64 + srow]) * sc;
        const size_t idx = (size_t)j * e.n + i;
        if (EPI == OZ_DOT) {  // conj(b) Y
          const double br = e.cur_re[idx], bi = e.cur_im[idx];
          dsr = fma(br, yr, fma(bi, yi, dsr));
          dsi = fma(br, yi, fma(-bi, yr, dsi));
        } else if (EPI == OZ_ADJ) {  // out = cpa g + i cw Y + b2
          const double gr = e.cur_re[idx], gi = e.cur_im[idx];
          double orr = e.cpa_re * gr - e.cpa_im * gi - e.cw * yi;
          double oi = e.cpa_re * gi + e.cpa_im * gr + e.cw * yr;
          if (e.prev_re) {
            orr += e.prev_re[idx];
            oi += e.prev_im[idx];
          }
          bad |= !(orr * orr + oi * oi <= tt.bound2);
          e.out_re[idx] = orr;
          e.out_im[idx] = oi;
        } else {  // Chebyshev term (as in the plain FP64 path)
          double pr, pi;
          if (tt.first) {
            pr = yi;
            pi = -yr;
          } else {
            pr = fma(2.0, yi, e.prev_re[idx]);
            pi = fma(-2.0, yr, e.prev_im[idx]);
          }
          bad |= !(pr * pr + pi * pi <= tt.bound2);
          double ar, ai;
          if (tt.first) {
            ar = fma(tt.coef, pr, tt.coef0 * e.cur_re[idx]);
            ai = fma(tt.coef, pi, tt.coef0 * e.cur_im[idx]);
          } else {
            ar = fma(tt.coef, pr, e.acc_re[idx]);
            ai = fma(tt.coef, pi, e.acc_im[idx]);
          }
          if (tt.last) {
            e.out_re[idx] = tt.ph_re * ar - tt.ph_im * ai;
            e.out_im[idx] = tt.ph_re * ai + tt.ph_im * ar;
          } else {
            e.out_re[idx] = pr;
            e.out_im[idx] = pi;
            e.acc_re[idx] = ar;
            e.acc_im[idx] = ai;
          }
        }
      }
      if (bad) atomicOr(tt.status, FQ_BIT_BOUND);
    }
    if (EPI == OZ_DOT) {  // per-CTA partial in a fixed order (bit-reproducible)
      double2* red = reinterpret_cast<double2*>(gbase + OZR_XS_BYTES);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        dsr += __shfl_xor_sync(0xffffffffu, dsr, o);
        dsi += __shfl_xor_sync(0xffffffffu, dsi, o);
      }
      if (lane == 0) red[warp - 2] = make_double2(dsr, dsi);
      asm volatile("bar.sync 1, %0;" ::"n"(32 * OZ_EPI_WARPS) : "memory");
      if (warp == 2 && lane == 0) {
        double sr = 0.0, si = 0.0;
        for (int q = 0; q < OZ_EPI_WARPS; ++q) {
          sr += red[q].x;
          si += red[q].y;
        }
        e.partial[tj * tiles_i + ti] = make_double2(sr, si);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS) : "memory");
  }
}

}  // namespace
