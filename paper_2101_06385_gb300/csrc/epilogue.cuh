// Epilogue of the single-accumulator tcgen05 squaring kernels (syrk_tc1.cu,
// syrk_tc2.cu).  Eight warps drain one 128 x 256 FP32 accumulator of
// 2^(2s) P = 2^(2s) Y^2 (Eq. 14) from TMEM and apply the layer of Alg. 1,
//     Y' = ca Y + cb P + cc I        (S = alpha I + Y, Eq. 16 form)
// with the diagonal in FP64 from the row norms (Y^2)_ii = sum_k Y_ik^2,
// re-split Y' into the FP16 operand planes of the next layer (Eq. 12: hp =
// 2^s hi and lo' for the split kernels, hi for plain FP16), store the
// upper tile and its mirror (only the upper tile of Y' when the launch keeps
// the iterate as a triangle, SqArgs::tri_y, and of the planes when it keeps
// them so, SqArgs::tri_planes), and publish the tile's FP64 (tr Y',
// ||Y'||_F^2) partial.
//
// Warp ew (0..7) owns TMEM lane quarter q (the warp's index mod 4, a
// hardware rule) and column half ew / 4: 32 rows x 128 columns, drained in
// four 32-column chunks (tcgen05.ld 32x32b: one row per lane).
//
// No named barrier is used: the eight per-warp partials of a tile meet in
// shared memory and the last warp to arrive (shared atomic counter) sums
// them in warp order, so the result does not depend on arrival order.  A
// partial slot is reused four tiles later; a warp can only reach that tile
// after every warp has released the accumulator two tiles after this one,
// which each warp does after it has finished this tile, so three slots would
// do.  A warp whose accumulator wait fails (time-out or abort) leaves
// without touching the barrier state of the others.
#pragma once

#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"
#include "tile_finish.cuh"

namespace sp2 {
namespace epi {

constexpr int WARPS = 8;
constexpr int SLOTS = 4;

// per-warp partials of a tile: tr Y', ||Y'||_F^2 and, in adjoint mode, the
// three dots (tr Yin, <Yin, aux>, <P, aux>)
constexpr int NRED = 5;

struct Shared {
  double red[SLOTS][WARPS][NRED];
  int cnt[SLOTS];
};

// thread 0, before the kernel's first __syncthreads
__device__ __forceinline__ void init(Shared& s) {
  for (int k = 0; k < SLOTS; ++k) s.cnt[k] = 0;
}

__device__ __forceinline__ uint32_t pack_h2(__half a, __half b) {
  return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
}

// (Y^2)_rr = sum_k Y_rk^2 of the input iterate: from the FP64 row norms, or
// summed in FP64 from the FP32 segment sums the previous launch left (eight
// accumulators over interleaved segments, combined in a fixed order).
__device__ __forceinline__ double row_norm(const SqArgs& a, int b, int N, int r) {
  if (!a.rnp_in) return a.rn ? a.rn[(long long)b * a.ld_rn + r] : 0.0;
  const float* p = a.rnp_in + (long long)b * a.slot_rnp + r;
  const int nseg = (N + 31) >> 5;
  double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  int s = 0;
  for (; s + 8 <= nseg; s += 8) {
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] += (double)p[(long long)(s + u) * a.ld_rnp];
  }
#pragma unroll
  for (int u = 0; u < 8; ++u)
    if (s + u < nseg) acc[u] += (double)p[(long long)(s + u) * a.ld_rnp];
  return ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
}

// Lane L returns sum over the 32 lanes of y[L]^2 (lanes with valid == false
// contribute zero): a butterfly that halves the values held per lane at each
// of the five exchange steps (31 shuffles).
__device__ __forceinline__ float column_sums_sq(const float (&y)[32], bool valid) {
  const int lane = threadIdx.x & 31;
  float s[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) s[j] = valid ? y[j] * y[j] : 0.f;
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) {
    const bool upper = (lane & w) != 0;
#pragma unroll
    for (int k = 0; k < w; ++k) {
      const float send = upper ? s[k] : s[k + w];
      const float keep = upper ? s[k + w] : s[k];
      s[k] = keep + __shfl_xor_sync(0xffffffffu, send, w);
    }
  }
  return s[0];
}

// Release of accumulator buffer buf by one lane of an epilogue warp.
template <bool PAIR>
__device__ __forceinline__ void release(uint64_t* tmem_empty, uint32_t buf, uint32_t empty_cl) {
  if (PAIR)
    sp2::tc::mbar_arrive_cl(empty_cl + 8u * buf);
  else
    sp2::tc::mbar_arrive(&tmem_empty[buf]);
}

// Tile t with accumulator use `it` (buffer it & 1).  Returns 0 when the
// tile's instance is inactive (nothing issued for it), 1 when done, -1 when
// the accumulator wait failed.
// ADJ (adjoint mode, a.aux set): the tile also accumulates, over its part
// of the full symmetric matrices, tr Yin, <Yin, aux> and <P, aux> on the
// old values, summed per instance into a.dots_out.
// RO (readout mode, a.R set): R += rc X' on the upper tiles, D = I - R in
// the launch that writes D (finite-temperature expansion).
// PAIR (CTA-pair kernels): the accumulator was written by the pair's MMA
// issuer in the even CTA, and the release of a buffer is an arrive on that
// CTA's barrier, empty_cl + 8 x buffer (a shared::cluster address).
template <bool SPLIT, bool ADJ = false, bool RO = false, bool PAIR = false>
__device__ __forceinline__ int tile(const SqArgs& a, int t, uint32_t it, uint32_t tmem_base, uint64_t* tmem_full,
                                    uint64_t* tmem_empty, volatile int* abort_flag, Shared& sh, int ew, int q,
                                    int lane, uint32_t empty_cl = 0u) {
  using namespace sp2::tc;
  int b, I, J, h;
  unpack_tile(a.tiles[t], b, I, J, h);
  const LayerParams p = load_params(a, b);
  if (!p.active) return 0;
  const int N = a.Ns[b];
  const int hc = ew >> 2;
  const int r = I * BN + h * BM + q * 32 + lane;
  const bool mirror = (I != J);
  const bool outD = (p.out_mode == OUT_D);
  // split: the accumulator holds 2^(2s) P (both operand planes scaled by 2^s)
  const float unscale = SPLIT ? a.lo_unscale * a.lo_unscale : 1.f;
  const float lo_scale = a.lo_scale;
  float* Y = a.Yout + (long long)b * a.slot_y;
  const float* Yold = a.Yin + (long long)b * a.slot_y;
  const long long ld = a.ld_y;

  // issued before the accumulator wait: the diagonal's FP64 row norm and
  // the old row segment (into L2)
  double rn_r = 0.0;
  if (r < N) {
    const int dcol = r - (J * BN + hc * 128);
    if (!mirror && (unsigned)dcol < 128u) rn_r = row_norm(a, b, N, r);
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
      const int c0 = J * BN + hc * 128 + ch * 32;
      if (c0 < N) asm volatile("prefetch.global.L2 [%0];" ::"l"(Yold + (long long)r * ld + c0));
    }
  }

  const uint32_t buf = it & 1u;
  const unsigned long long lim = wait_limit(a);
  const bool got = __all_sync(0xffffffffu, PAIR ? mbar_wait_cl(&tmem_full[buf], (it >> 1) & 1u, abort_flag, lim)
                                                : mbar_wait(&tmem_full[buf], (it >> 1) & 1u, abort_flag, lim));
  if (!got) {
    if (lane == 0) atomicExch(a.err, (int)SP2_ERR_DEVICE_TIMEOUT);
    *abort_flag = 1;
    return -1;
  }
  tc_fence_after();

  float* rnp = a.rnp_out ? a.rnp_out + (long long)b * a.slot_rnp : nullptr;
  __half* ho = a.hi_out ? a.hi_out + (long long)b * a.slot_h : nullptr;
  __half* lo_ = a.lo_out ? a.lo_out + (long long)b * a.slot_h : nullptr;
  __half* hp_ = a.hp_out ? a.hp_out + (long long)b * a.slot_h : nullptr;
  // the plane scaled like the accumulator's operands: hp for split, hi for plain
  __half* const pa_out = SPLIT ? hp_ : ho;
  const long long ldh = a.ld_h;
  float* D = outD ? a.Dptr[b] : nullptr;
  double tr = 0.0, sq = 0.0;
  // adjoint-mode dots; dtr carries the Tr[D A] partial in the launch that writes D
  double dtr = 0.0, dgy = 0.0, dpy = 0.0;
  const uint32_t taddr = tmem_base + buf * BN + ((uint32_t)(q * 32) << 16) + hc * 128;
  const bool vec_y = (ld & 3) == 0;

  // chunks wholly past the padded K extent (columns >= round_up(N, 64)) or
  // warps whose 32 rows all lie past N have nothing to write (warp-uniform)
  const int kpad = (N + 63) & ~63;
  const bool rows_live = I * BN + h * BM + q * 32 < N;

#pragma unroll 1
  for (int ch = 0; ch < 4; ++ch) {
    const int c0 = J * BN + hc * 128 + ch * 32;
    if (!rows_live || c0 >= kpad) {
      if (ch == 3) {
        tc_fence_before();
        __syncwarp();
        if (lane == 0) release<PAIR>(tmem_empty, buf, empty_cl);
      }
      continue;
    }
    // the diagonal element of row r, if it lies in this chunk (I == J only)
    const int jd = r - c0;
    const bool dchunk = !mirror && (unsigned)jd < 32u;
    const bool full_chunk = (c0 + 32 <= N) && vec_y;
    // old values first: their global-load latency overlaps the TMEM load
    float y[32];
    if (r >= N) {
#pragma unroll
      for (int j = 0; j < 32; ++j) y[j] = 0.f;
    } else if (full_chunk) {
      const float4* src = reinterpret_cast<const float4*>(Yold + (long long)r * ld + c0);
#pragma unroll
      for (int j4 = 0; j4 < 8; ++j4) {
        const float4 o = src[j4];
        y[4 * j4 + 0] = o.x;
        y[4 * j4 + 1] = o.y;
        y[4 * j4 + 2] = o.z;
        y[4 * j4 + 3] = o.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) y[j] = (c0 + j < N) ? Yold[(long long)r * ld + c0 + j] : 0.f;
    }
    uint32_t v[32];
    const bool packs = !outD && r < N && (pa_out || lo_) && c0 + 32 <= (int)ldh;
    __syncwarp();
    tmem_ld32(taddr + ch * 32, v);
    tmem_ld_wait();
    if (ch == 3) {
      // accumulator drained: the MMA issuer may reuse this buffer
      tc_fence_before();
      __syncwarp();
      if (lane == 0) release<PAIR>(tmem_empty, buf, empty_cl);
    }
    if (r < N) {
      float yold_d = 0.f, p_d = 0.f;
      if (dchunk) {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (j == jd) {
            yold_d = y[j];
            p_d = __uint_as_float(v[j]) * unscale;
          }
      }
      if (ADJ) {
        // dots on the old values (before the update overwrites y)
        const float* ax = a.aux + (long long)b * a.slot_y + (long long)r * ld + c0;
        float gy = 0.f, py = 0.f;
#pragma unroll
        for (int j4 = 0; j4 < 8; ++j4) {
          float x[4];
          if (full_chunk) {
            const float4 o = reinterpret_cast<const float4*>(ax)[j4];
            x[0] = o.x;
            x[1] = o.y;
            x[2] = o.z;
            x[3] = o.w;
          } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = (c0 + 4 * j4 + u < N) ? ax[4 * j4 + u] : 0.f;
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = 4 * j4 + u;
            gy = fmaf(y[j], x[u], gy);
            py = fmaf(__uint_as_float(v[j]) * unscale, x[u], py);
          }
        }
        dgy += (double)gy;
        dpy += (double)py;
        if (dchunk) dtr += (double)yold_d;
      }
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const float P = __uint_as_float(v[j]) * unscale;
        const float yn = fmaf(p.ca, y[j], p.cb * P);
        y[j] = (c0 + j < N) ? yn : 0.f;
      }
      // one FP64 update per row, outside the unrolled element loop
      float ydo = 0.f;
      double yd = 0.0;
      if (dchunk) {
        const double pd = (a.rn || a.rnp_in) ? rn_r : (double)p_d;
        yd = p.ca_d * (double)yold_d + p.cb_d * pd + p.cc_d;
        tr += yd;
        const float ydf = (float)yd;
        ydo = outD ? (float)(yd + p.alpha_out) : ydf;
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (j == jd) y[j] = ydf;
      }
      float sqf = 0.f;
#pragma unroll
      for (int j = 0; j < 32; ++j) sqf = fmaf(y[j], y[j], sqf);
      sq += (double)sqf;
      if (rnp && c0 < N) rnp[(long long)(c0 >> 5) * a.ld_rnp + r] = sqf;
      if (RO) {
        // readout R += rc X' over the upper tiles (R is symmetric; its lower
        // half is only needed as D, written with the mirror below); two
        // halves of 16 columns keep the register footprint down
        float* Rr = a.R + (long long)b * a.slot_y + (long long)r * ld + c0;
        double rd = 0.0;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          float rv[16];
          if (full_chunk) {
#pragma unroll
            for (int j4 = 0; j4 < 4; ++j4) {
              const float4 o = reinterpret_cast<const float4*>(Rr + 16 * hh)[j4];
              rv[4 * j4 + 0] = o.x;
              rv[4 * j4 + 1] = o.y;
              rv[4 * j4 + 2] = o.z;
              rv[4 * j4 + 3] = o.w;
            }
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) rv[j] = (c0 + 16 * hh + j < N) ? Rr[16 * hh + j] : 0.f;
          }
          const bool dhalf = dchunk && (jd >> 4) == hh;
          if (dhalf) {
            float rold = 0.f;
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (16 * hh + j == jd) rold = rv[j];
            rd = (double)rold + p.rc_d * (yd + p.alpha_new);
          }
#pragma unroll
          for (int j = 0; j < 16; ++j) rv[j] = fmaf(p.rc, y[16 * hh + j], rv[j]);
          if (dhalf) {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (16 * hh + j == jd) rv[j] = (float)rd;
          }
          if (outD) {
            // D = I - R: the values the D stores (and the mirror) write
#pragma unroll
            for (int j = 0; j < 16; ++j) y[16 * hh + j] = (c0 + 16 * hh + j < N) ? -rv[j] : 0.f;
          } else if (full_chunk) {
#pragma unroll
            for (int j4 = 0; j4 < 4; ++j4)
              reinterpret_cast<float4*>(Rr + 16 * hh)[j4] =
                  make_float4(rv[4 * j4], rv[4 * j4 + 1], rv[4 * j4 + 2], rv[4 * j4 + 3]);
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (c0 + 16 * hh + j < N) Rr[16 * hh + j] = rv[j];
          }
        }
        if (outD) ydo = (float)(1.0 - rd);
      }
      if (outD) {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (c0 + j < N) D[(long long)r * N + c0 + j] = (dchunk && j == jd) ? ydo : y[j];
        if (!ADJ && a.Hobs) {
          // Tr[D A] over this row segment (A symmetric: the mirror counts twice below)
          const float* hr = a.Hobs[b] + (long long)r * N + c0;
          const bool hvec = ((N & 3) == 0) && (c0 + 32 <= N) && ((((uintptr_t)a.Hobs[b]) & 15) == 0);
          float eo = 0.f;
#pragma unroll
          for (int j4 = 0; j4 < 8; ++j4) {
            float x[4];
            if (hvec) {
              const float4 o = reinterpret_cast<const float4*>(hr)[j4];
              x[0] = o.x;
              x[1] = o.y;
              x[2] = o.z;
              x[3] = o.w;
            } else {
#pragma unroll
              for (int u = 0; u < 4; ++u) x[u] = (c0 + 4 * j4 + u < N) ? hr[4 * j4 + u] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int j = 4 * j4 + u;
              eo = fmaf((dchunk && j == jd) ? ydo : y[j], x[u], eo);
            }
          }
          dtr += (double)eo;
        }
      } else {
        if (full_chunk) {
          float4* dst = reinterpret_cast<float4*>(Y + (long long)r * ld + c0);
#pragma unroll
          for (int j4 = 0; j4 < 8; ++j4) dst[j4] = make_float4(y[4 * j4], y[4 * j4 + 1], y[4 * j4 + 2], y[4 * j4 + 3]);
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (c0 + j < N) Y[(long long)r * ld + c0 + j] = y[j];
        }
      }
    }
    // row norms of the mirror: rows c0 + j of Y' get the segment of the 32
    // rows of this warp, the column sums of y^2 over the lanes
    if (mirror && rnp) {
      const float cs = column_sums_sq(y, r < N);
      if (c0 + lane < N) rnp[(long long)((I * BN + h * BM + q * 32) >> 5) * a.ld_rnp + c0 + lane] = cs;
    }
    // mirrored store: lanes hold consecutive rows r -> consecutive columns
    if (mirror && r < N && (outD || !a.tri_y)) {
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int c = c0 + j;
        if (c < N) {
          if (outD)
            D[(long long)c * N + r] = y[j];
          else
            Y[(long long)c * ld + r] = y[j];
        }
      }
    }
    if (packs) {
      // FP16 planes of Y': 32 halves per plane packed in registers, stored
      // to the row segment and (off-diagonal tiles) its mirror; columns >= N
      // carry zeros
      uint32_t pa[16], pl[16];  // hp (split) or hi (plain), and lo'
#pragma unroll
      for (int j2 = 0; j2 < 16; ++j2) {
        __half h0, l0, h1, l1;
        split_fp16(y[2 * j2], lo_scale, h0, l0);
        split_fp16(y[2 * j2 + 1], lo_scale, h1, l1);
        pa[j2] = SPLIT ? pack_h2(__float2half_rn(__half2float(h0) * lo_scale),
                                 __float2half_rn(__half2float(h1) * lo_scale))
                       : pack_h2(h0, h1);
        pl[j2] = pack_h2(l0, l1);
      }
      if (pa_out) {
        uint4* dp = reinterpret_cast<uint4*>(pa_out + (long long)r * ldh + c0);
#pragma unroll
        for (int j4 = 0; j4 < 4; ++j4) dp[j4] = make_uint4(pa[4 * j4], pa[4 * j4 + 1], pa[4 * j4 + 2], pa[4 * j4 + 3]);
      }
      if (lo_) {
        uint4* dl = reinterpret_cast<uint4*>(lo_ + (long long)r * ldh + c0);
#pragma unroll
        for (int j4 = 0; j4 < 4; ++j4) dl[j4] = make_uint4(pl[4 * j4], pl[4 * j4 + 1], pl[4 * j4 + 2], pl[4 * j4 + 3]);
      }
      if (mirror && !a.tri_planes) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int c = c0 + j;
          if (c < N) {
            const int sh16 = 16 * (j & 1);
            if (pa_out) pa_out[(long long)c * ldh + r] = __ushort_as_half((unsigned short)(pa[j >> 1] >> sh16));
            if (lo_) lo_[(long long)c * ldh + r] = __ushort_as_half((unsigned short)(pl[j >> 1] >> sh16));
          }
        }
      }
    }
  }

  const bool energy = !ADJ && outD && a.Hobs;  // dtr holds the Tr[D A] partial
  if (mirror) {
    sq *= 2.0;
    dgy *= 2.0;
    dpy *= 2.0;
    if (energy) dtr *= 2.0;
  }
  tr = warp_sum_d(tr);
  sq = warp_sum_d(sq);
  if (ADJ || energy) {
    dtr = warp_sum_d(dtr);
    dgy = warp_sum_d(dgy);
    dpy = warp_sum_d(dpy);
  }
  const int slot = (int)(it & (SLOTS - 1));
  unsigned last = 0;
  if (lane == 0) {
    sh.red[slot][ew][0] = tr;
    sh.red[slot][ew][1] = sq;
    sh.red[slot][ew][2] = dtr;
    sh.red[slot][ew][3] = dgy;
    sh.red[slot][ew][4] = dpy;
    __threadfence_block();
    last = (atomicAdd(&sh.cnt[slot], 1) == WARPS - 1) ? 1u : 0u;
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (last) {
    __threadfence_block();
    double T = 0.0, Q = 0.0;
    if (lane == 0) {
      volatile double* rd = &sh.red[slot][0][0];
      double d0 = 0.0, d1 = 0.0, d2 = 0.0;
      for (int k = 0; k < WARPS; ++k) {
        T += rd[NRED * k];
        Q += rd[NRED * k + 1];
        d0 += rd[NRED * k + 2];
        d1 += rd[NRED * k + 3];
        d2 += rd[NRED * k + 4];
      }
      if (ADJ || energy) {
        a.tile_dots[3 * (long long)t + 0] = d0;
        a.tile_dots[3 * (long long)t + 1] = d1;
        a.tile_dots[3 * (long long)t + 2] = d2;
      }
      sh.cnt[slot] = 0;
    }
    finish_tile_warp(a, t, b, T, Q, p.out_mode);
  }
  return 1;
}

}  // namespace epi
}  // namespace sp2
