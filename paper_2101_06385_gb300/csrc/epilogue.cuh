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
// four 32-column chunks (tcgen05.ld 32x32b: one row per lane).  Each chunk is
// turned through a 4 KB shared-memory buffer of the warp so that a lane holds
// four consecutive columns of eight rows: the loads and stores of the
// iterate, the planes and the other row-major operands then cover whole
// 128-byte row segments.
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

// A tile's sums handed from the epilogue warps to the finisher warp, which
// publishes them and, for the last tile of an instance, runs its control
// step (off the epilogue warps' path: that work is a chain of global
// round trips).
constexpr int FQ = 4;
struct FinEntry {
  int t, b, out_mode, dots;
  double T, Q, d0, d1, d2;
};

struct Shared {
  double red[SLOTS][WARPS][NRED];
  int cnt[SLOTS];
  FinEntry fq[FQ];
  uint64_t fin_full[FQ];   // entry written (one arrive)
  uint64_t fin_empty[FQ];  // entry read by the finisher (one arrive)
};

// thread 0, before the kernel's mbarrier-init fence and first __syncthreads
__device__ __forceinline__ void init(Shared& s) {
  for (int k = 0; k < SLOTS; ++k) s.cnt[k] = 0;
  for (int k = 0; k < FQ; ++k) {
    sp2::tc::mbar_init(&s.fin_full[k], 1);
    sp2::tc::mbar_init(&s.fin_empty[k], 1);
  }
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

// Release of accumulator buffer buf by one lane of an epilogue warp.
template <bool PAIR>
__device__ __forceinline__ void release(uint64_t* tmem_empty, uint32_t buf, uint32_t empty_cl) {
  if (PAIR)
    sp2::tc::mbar_arrive_cl(empty_cl + 8u * buf);
  else
    sp2::tc::mbar_arrive(&tmem_empty[buf]);
}

// The warp's staging buffer in shared memory holds one 32 x 32 FP32 chunk,
// row r at r * 32 floats, its 16-byte group m (columns 4m .. 4m + 3) at group
// m ^ (r & 7).  A warp writing one row per lane, or reading four rows with
// eight lanes each, touches every bank once per 128 bytes: four wavefronts
// per 512-byte access, the least there can be.
constexpr int TR_FLOATS = 32 * 32;
constexpr int TR_BYTES = WARPS * TR_FLOATS * 4;  // per CTA: 32 KB

__device__ __forceinline__ float4* tr_at(float* trb, int r, int m) {
  return reinterpret_cast<float4*>(trb + r * 32 + ((m ^ (r & 7)) << 2));
}

// Four consecutive floats of a row, columns c .. c + 3 at p (zeros at and
// past column n); one 16-byte access when vec (16-byte aligned rows) and the
// four are inside.
__device__ __forceinline__ float4 ld4(const float* p, int c, int n, bool vec) {
  if (vec && c + 4 <= n) return *reinterpret_cast<const float4*>(p);
  float4 r;
  r.x = c < n ? p[0] : 0.f;
  r.y = c + 1 < n ? p[1] : 0.f;
  r.z = c + 2 < n ? p[2] : 0.f;
  r.w = c + 3 < n ? p[3] : 0.f;
  return r;
}
__device__ __forceinline__ void st4(float* p, float4 v, int c, int n, bool vec) {
  if (vec && c + 4 <= n) {
    *reinterpret_cast<float4*>(p) = v;
    return;
  }
  if (c < n) p[0] = v.x;
  if (c + 1 < n) p[1] = v.y;
  if (c + 2 < n) p[2] = v.z;
  if (c + 3 < n) p[3] = v.w;
}

// Sums over the N_ lanes that differ only in lane bits LOWBIT .. LOWBIT +
// log2(N_) - 1: each of them holds N_ values s[0 .. N_), and a lane returns
// the total over those lanes of value index (lane >> LOWBIT) & (N_ - 1).  A
// halving butterfly (N_ - 1 shuffles); s is overwritten.
template <int N_, int LOWBIT>
__device__ __forceinline__ float lane_sums(float (&s)[N_]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int w = N_ / 2; w >= 1; w >>= 1) {
    const bool upper = ((lane >> LOWBIT) & w) != 0;
#pragma unroll
    for (int k = 0; k < w; ++k) {
      const float send = upper ? s[k] : s[k + w];
      const float keep = upper ? s[k + w] : s[k];
      s[k] = keep + __shfl_xor_sync(0xffffffffu, send, w << LOWBIT);
    }
  }
  return s[0];
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
//
// Layout of the work: a chunk is the warp's 32 accumulator rows x 32 columns
// (lane = row after tcgen05.ld).  Through the staging buffer trb, lane
// (r4, c4) = (lane / 8, lane % 8) takes columns c0 + 4 c4 .. + 3 of the
// eight rows R0 + 4 i + r4 (registers 4 i .. 4 i + 3).  Every warp
// instruction that loads or stores the iterate, the operand planes, H, R or
// aux then covers four whole 128-byte row segments.  Stores of the mirror
// block go back through the buffer to the row-per-lane layout, where they
// are contiguous too.
template <bool SPLIT, bool ADJ = false, bool RO = false, bool PAIR = false>
__device__ __forceinline__ int tile(const SqArgs& a, int t, uint32_t it, uint32_t tmem_base, uint64_t* tmem_full,
                                    uint64_t* tmem_empty, volatile int* abort_flag, Shared& sh, int ew, int q,
                                    int lane, float* trb, uint32_t empty_cl = 0u) {
  using namespace sp2::tc;
  int b, I, J, h;
  unpack_tile(a.tiles[t], b, I, J, h);
  const LayerParams p = load_params(a, b);
  if (!p.active) return 0;
  const int N = a.Ns[b];
  const int hc = ew >> 2;
  const int R0 = I * BN + h * BM + q * 32;  // first of the warp's 32 rows
  const int nrows = min(32, N - R0);        // rows of the warp inside the matrix (may be <= 0)
  const bool mirror = (I != J);
  const bool outD = (p.out_mode == OUT_D);
  // split: the accumulator holds 2^(2s) P (both operand planes scaled by 2^s)
  const float unscale = SPLIT ? a.lo_unscale * a.lo_unscale : 1.f;
  const float lo_scale = a.lo_scale;
  float* Y = a.Yout + (long long)b * a.slot_y;
  const float* Yold = a.Yin + (long long)b * a.slot_y;
  const long long ld = a.ld_y;
  const int cbase = J * BN + hc * 128;      // first column of the warp's half
  const int r4 = lane >> 3, c4 = lane & 7;

  // issued before the accumulator wait: the FP64 row norm of the diagonal
  // element this lane will hold (row R0 + 4 c4 + r4, in the chunk whose first
  // column is R0) and the warp's old rows (into L2)
  double rn_l = 0.0;
  const int rdiag = R0 + 4 * c4 + r4;
  const bool dwarp = !mirror && (unsigned)(R0 - cbase) < 128u;  // the warp's columns hold its diagonal
  if (dwarp && rdiag < N) rn_l = row_norm(a, b, N, rdiag);
  if (lane < nrows) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int c0 = cbase + c * 32;
      if (c0 < N) asm volatile("prefetch.global.L2 [%0];" ::"l"(Yold + (long long)(R0 + lane) * ld + c0));
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
  // 16-byte accesses where every row start of the matrix is 16-byte aligned:
  // Y, Y_old (and R, aux) with leading dimension ld; D and H with N
  const float* Rb0 = RO ? a.R + (long long)b * a.slot_y : nullptr;
  const float* Xb0 = ADJ ? a.aux + (long long)b * a.slot_y : nullptr;
  const bool vec_y = (ld & 3) == 0 &&
                     ((reinterpret_cast<uintptr_t>(Y) | reinterpret_cast<uintptr_t>(Yold) |
                       reinterpret_cast<uintptr_t>(Rb0) | reinterpret_cast<uintptr_t>(Xb0)) & 15) == 0;
  const float* Hb0 = (outD && !ADJ && a.Hobs) ? a.Hobs[b] : nullptr;
  const bool vec_n = (N & 3) == 0 &&
                     ((reinterpret_cast<uintptr_t>(D) | reinterpret_cast<uintptr_t>(Hb0)) & 15) == 0;
  double tr = 0.0, sq = 0.0;
  // adjoint-mode dots; dtr carries the Tr[D A] partial in the launch that writes D
  double dtr = 0.0, dgy = 0.0, dpy = 0.0;
  const uint32_t taddr = tmem_base + buf * BN + ((uint32_t)(q * 32) << 16) + hc * 128;

  // chunks wholly past the padded K extent (columns >= round_up(N, 64)) or
  // warps whose 32 rows all lie past N have nothing to write (warp-uniform)
  const int kpad = (N + 63) & ~63;
  const bool rows_live = nrows > 0;
  // mirror blocks stored in this launch (off-diagonal tiles only)
  const bool mir_y = mirror && (outD || !a.tri_y);
  const bool mir_p = mirror && !outD && !a.tri_planes && (pa_out || lo_);

#pragma unroll 1
  for (int ch = 0; ch < 4; ++ch) {
    const int c0 = cbase + ch * 32;
    if (!rows_live || c0 >= kpad) {
      if (ch == 3) {
        tc_fence_before();
        __syncwarp();
        if (lane == 0) release<PAIR>(tmem_empty, buf, empty_cl);
      }
      continue;
    }
    const int ce = c0 + 4 * c4;  // this lane's first column
    // the one diagonal element a lane holds (chunk c0 == R0 of a diagonal
    // tile, a warp-uniform condition): row = column = rdiag, register 4 c4 + r4
    const bool dchunk = !mirror && c0 == R0;
    const bool dlane = dchunk && rdiag < N;
    const int id = 4 * c4 + r4;
    // every row and column of the chunk inside the matrix (warp-uniform)
    const bool full = nrows == 32 && c0 + 32 <= N;
    // old values first: their global-load latency overlaps the TMEM load
    float y[32];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const bool rok = 4 * i + r4 < nrows;
      const float4 o = rok ? ld4(Yold + (long long)(R0 + 4 * i + r4) * ld + ce, ce, N, vec_y)
                           : make_float4(0.f, 0.f, 0.f, 0.f);
      y[4 * i] = o.x;
      y[4 * i + 1] = o.y;
      y[4 * i + 2] = o.z;
      y[4 * i + 3] = o.w;
    }
    {
      uint32_t v[32];
      __syncwarp();
      tmem_ld32(taddr + ch * 32, v);
      tmem_ld_wait();
      if (ch == 3) {
        // accumulator drained: the MMA issuer may reuse this buffer
        tc_fence_before();
        __syncwarp();
        if (lane == 0) release<PAIR>(tmem_empty, buf, empty_cl);
      }
      // lane = row -> lane = (four rows, four columns)
#pragma unroll
      for (int m = 0; m < 8; ++m)
        *tr_at(trb, lane, m) = make_float4(__uint_as_float(v[4 * m]), __uint_as_float(v[4 * m + 1]),
                                           __uint_as_float(v[4 * m + 2]), __uint_as_float(v[4 * m + 3]));
    }
    __syncwarp();
    // the diagonal element's old value and product (diagonal chunks only;
    // P(4 c4 + r4, 4 c4 + r4) sits in this lane's row group c4, component r4)
    float yold_d = 0.f, p_d = 0.f;
    if (dchunk) {
#pragma unroll
      for (int k = 0; k < 32; ++k)
        if (k == id) yold_d = y[k];
      const float4 pdv = *tr_at(trb, 4 * c4 + r4, c4);
      p_d = (r4 == 0 ? pdv.x : r4 == 1 ? pdv.y : r4 == 2 ? pdv.z : pdv.w) * unscale;
    }
    {
      // cb * unscale is exact (a power of two): y' = ca y + (cb 2^-2s) P_acc
      const float cbu = p.cb * unscale;
      float gy = 0.f, py = 0.f;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float4 pv = *tr_at(trb, 4 * i + r4, c4);
        const float P[4] = {pv.x, pv.y, pv.z, pv.w};
        if (ADJ) {
          // dots on the old values (before the update overwrites y)
          float x[4] = {0.f, 0.f, 0.f, 0.f};
          if (4 * i + r4 < nrows) {
            const float4 xv =
                ld4(a.aux + (long long)b * a.slot_y + (long long)(R0 + 4 * i + r4) * ld + ce, ce, N, vec_y);
            x[0] = xv.x;
            x[1] = xv.y;
            x[2] = xv.z;
            x[3] = xv.w;
          }
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            gy = fmaf(y[4 * i + e], x[e], gy);
            py = fmaf(P[e] * unscale, x[e], py);
          }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) y[4 * i + e] = fmaf(p.ca, y[4 * i + e], cbu * P[e]);
      }
      if (!full) {
        // rows past nrows and columns past N stay zero
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (!(4 * i + r4 < nrows && ce + e < N)) y[4 * i + e] = 0.f;
      }
      if (ADJ) {
        dgy += (double)gy;
        dpy += (double)py;
        if (dlane) dtr += (double)yold_d;
      }
    }
    __syncwarp();
    // one FP64 update per diagonal element, outside the unrolled element loop
    float ydo = 0.f;
    double yd = 0.0;
    if (dchunk) {
      if (dlane) {
        const double pd = (a.rn || a.rnp_in) ? rn_l : (double)p_d;
        yd = p.ca_d * (double)yold_d + p.cb_d * pd + p.cc_d;
        tr += yd;
        ydo = outD ? (float)(yd + p.alpha_out) : (float)yd;
      }
      const float ydf = (float)yd;
#pragma unroll
      for (int k = 0; k < 32; ++k)
        if (dlane && k == id) y[k] = ydf;
    }
    // sums of squares of Y': per row (over the chunk's 32 columns) and per
    // column (over the warp's 32 rows), and this lane's share of ||Y'||_F^2
    float rs[8], cs[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      rs[i] = 0.f;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        rs[i] = fmaf(y[4 * i + e], y[4 * i + e], rs[i]);
        cs[e] = fmaf(y[4 * i + e], y[4 * i + e], cs[e]);
      }
    }
    sq += (double)(((rs[0] + rs[1]) + (rs[2] + rs[3])) + ((rs[4] + rs[5]) + (rs[6] + rs[7])));
    if (rnp) {
      // row R0 + 4 c4 + r4, segment c0 / 32; and for the mirror, row
      // c0 + 4 c4 + r4 (a column here), segment R0 / 32
      const float rsum = lane_sums<8, 0>(rs);
      if (rdiag < N && c0 < N) rnp[(long long)(c0 >> 5) * a.ld_rnp + rdiag] = rsum;
      if (mirror) {
        const float csum = lane_sums<4, 3>(cs);
        const int cm = c0 + 4 * c4 + r4;
        if (cm < N) rnp[(long long)(R0 >> 5) * a.ld_rnp + cm] = csum;
      }
    }
    if (RO) {
      // readout R += rc X' over the upper tiles (R is symmetric; its lower
      // half is only needed as D, written with the mirror below); all loads
      // before the first store (the compiler cannot tell the rows apart)
      // (rows in two halves of four, to bound the registers held)
      float* Rb = a.R + (long long)b * a.slot_y + (long long)R0 * ld + ce;
      double rd = 0.0;
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        float4 rv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = 4 * hh + u;
          rv[u] = (4 * i + r4 < nrows) ? ld4(Rb + (long long)(4 * i + r4) * ld, ce, N, vec_y)
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        // register id = 4 c4 + r4: row group c4, component r4
        if (dlane && (c4 >> 2) == hh) {
          float rold = 0.f;
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (4 * hh + u == c4) rold = r4 == 0 ? rv[u].x : r4 == 1 ? rv[u].y : r4 == 2 ? rv[u].z : rv[u].w;
          rd = (double)rold + p.rc_d * (yd + p.alpha_new);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = 4 * hh + u;
          const bool rok = 4 * i + r4 < nrows;
          float r_[4] = {rv[u].x, rv[u].y, rv[u].z, rv[u].w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int k = 4 * i + e;
            r_[e] = fmaf(p.rc, y[k], r_[e]);
            if (dlane && k == id) r_[e] = (float)rd;
            if (outD) y[k] = (rok && ce + e < N) ? -r_[e] : 0.f;  // D = I - R
          }
          if (!outD && rok)
            st4(Rb + (long long)(4 * i + r4) * ld, make_float4(r_[0], r_[1], r_[2], r_[3]), ce, N, vec_y);
        }
      }
      if (outD) ydo = (float)(1.0 - rd);
    }
    if (outD) {
      // D's diagonal: alpha + Y'_ii in FP64, rounded once
      if (dchunk) {
#pragma unroll
        for (int k = 0; k < 32; ++k)
          if (dlane && k == id) y[k] = ydo;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (4 * i + r4 < nrows)
          st4(D + (long long)(R0 + 4 * i + r4) * N + ce, make_float4(y[4 * i], y[4 * i + 1], y[4 * i + 2], y[4 * i + 3]),
              ce, N, vec_n);
      }
      if (!ADJ && a.Hobs) {
        // Tr[D A] over this chunk (A symmetric: the mirror counts twice below)
        float eo = 0.f;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          if (4 * i + r4 < nrows) {
            const float4 hv = ld4(a.Hobs[b] + (long long)(R0 + 4 * i + r4) * N + ce, ce, N, vec_n);
            const float hx[4] = {hv.x, hv.y, hv.z, hv.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) eo = fmaf(y[4 * i + e], hx[e], eo);
          }
        }
        dtr += (double)eo;
      }
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (4 * i + r4 < nrows)
          st4(Y + (long long)(R0 + 4 * i + r4) * ld + ce, make_float4(y[4 * i], y[4 * i + 1], y[4 * i + 2], y[4 * i + 3]),
              ce, N, vec_y);
    }
    // FP16 planes of Y' (Eq. 12): the row segments, four halves per plane and
    // lane (columns up to the padded row length carry zeros)
    if (!outD && (pa_out || lo_) && c0 + 32 <= (int)ldh) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (4 * i + r4 < nrows) {
          // Eq. 12 on pairs of elements: hi = fp16(x), lo' = fp16(2^s (x - hi));
          // hp = 2^s hi is exact in FP16 (|x| < 16), so one packed multiply
          uint32_t pa[2], pl[2];
          const __half2 s2 = __float2half2_rn(lo_scale);
#pragma unroll
          for (int e2 = 0; e2 < 2; ++e2) {
            const float x0 = y[4 * i + 2 * e2], x1 = y[4 * i + 2 * e2 + 1];
            const __half2 h2 = __floats2half2_rn(x0, x1);
            const float2 hf = __half22float2(h2);
            const __half2 l2 = __floats2half2_rn((x0 - hf.x) * lo_scale, (x1 - hf.y) * lo_scale);
            const __half2 p2 = SPLIT ? __hmul2(h2, s2) : h2;
            pa[e2] = *reinterpret_cast<const uint32_t*>(&p2);
            pl[e2] = *reinterpret_cast<const uint32_t*>(&l2);
          }
          const long long off = (long long)(R0 + 4 * i + r4) * ldh + ce;
          if (pa_out) *reinterpret_cast<uint2*>(pa_out + off) = make_uint2(pa[0], pa[1]);
          if (lo_) *reinterpret_cast<uint2*>(lo_ + off) = make_uint2(pl[0], pl[1]);
        }
      }
    }
    if (mir_y || mir_p) {
      // back to lane = row: lane L holds (row R0 + L, column c0 + k) in y[k],
      // and the mirror element (c0 + k, R0 + L) is contiguous across lanes
#pragma unroll
      for (int i = 0; i < 8; ++i)
        *tr_at(trb, 4 * i + r4, c4) = make_float4(y[4 * i], y[4 * i + 1], y[4 * i + 2], y[4 * i + 3]);
      __syncwarp();
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const float4 o = *tr_at(trb, lane, m);
        y[4 * m] = o.x;
        y[4 * m + 1] = o.y;
        y[4 * m + 2] = o.z;
        y[4 * m + 3] = o.w;
      }
      __syncwarp();
      if (lane < nrows) {
        const int r = R0 + lane;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          const int c = c0 + k;
          if (c < N) {
            if (mir_y) {
              if (outD)
                D[(long long)c * N + r] = y[k];
              else
                Y[(long long)c * ld + r] = y[k];
            }
            if (mir_p) {
              __half hh, ll;
              split_fp16(y[k], lo_scale, hh, ll);
              if (pa_out) pa_out[(long long)c * ldh + r] = SPLIT ? __float2half_rn(__half2float(hh) * lo_scale) : hh;
              if (lo_) lo_[(long long)c * ldh + r] = ll;
            }
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
  if (last && lane == 0) {
    // the last warp of the tile sums the partials in warp order and hands
    // them to the finisher warp (entry `it` of its queue)
    __threadfence_block();
    volatile double* rd = &sh.red[slot][0][0];
    double T = 0.0, Q = 0.0, d0 = 0.0, d1 = 0.0, d2 = 0.0;
    for (int k = 0; k < WARPS; ++k) {
      T += rd[NRED * k];
      Q += rd[NRED * k + 1];
      d0 += rd[NRED * k + 2];
      d1 += rd[NRED * k + 3];
      d2 += rd[NRED * k + 4];
    }
    sh.cnt[slot] = 0;
    const uint32_t e = it % FQ;
    if (mbar_wait(&sh.fin_empty[e], ((it / FQ) & 1u) ^ 1u, abort_flag, lim)) {
      FinEntry& f = sh.fq[e];
      f.t = t;
      f.b = b;
      f.out_mode = p.out_mode;
      f.dots = (ADJ || energy) ? 1 : 0;
      f.T = T;
      f.Q = Q;
      f.d0 = d0;
      f.d1 = d1;
      f.d2 = d2;
      mbar_arrive(&sh.fin_full[e]);
    } else {
      atomicExch(a.err, (int)SP2_ERR_DEVICE_TIMEOUT);
    }
  }
  return 1;
}

// The finisher warp's work for one active tile: waits for the tile's entry
// (the it-th of the CTA), writes its per-tile sums and runs
// finish_tile_warp (the instance's control step after its last tile).
// False on an abort.
__device__ __forceinline__ bool finish_entry(const SqArgs& a, uint32_t it, Shared& sh, volatile int* abort_flag,
                                             int lane, unsigned long long lim) {
  using namespace sp2::tc;
  const uint32_t e = it % FQ;
  if (!__all_sync(0xffffffffu, mbar_wait(&sh.fin_full[e], (it / FQ) & 1u, abort_flag, lim))) {
    if (lane == 0) atomicExch(a.err, (int)SP2_ERR_DEVICE_TIMEOUT);
    *abort_flag = 1;
    return false;
  }
  const FinEntry f = sh.fq[e];
  if (lane == 0 && f.dots) {
    a.tile_dots[3 * (long long)f.t + 0] = f.d0;
    a.tile_dots[3 * (long long)f.t + 1] = f.d1;
    a.tile_dots[3 * (long long)f.t + 2] = f.d2;
  }
  __syncwarp();
  if (lane == 0) mbar_arrive(&sh.fin_empty[e]);
  finish_tile_warp(a, f.t, f.b, f.T, f.Q, f.out_mode);
  return true;
}

// The finisher warp: for every active tile of the CTA, in the order the
// epilogue warps take them (tile(t) for t = first, first + stride, ...),
// finish_entry.  Returns early on an abort.
__device__ __forceinline__ void finisher(const SqArgs& a, int first, int stride, int count, Shared& sh,
                                         volatile int* abort_flag, int lane) {
  using namespace sp2::tc;
  const unsigned long long lim = wait_limit(a);
  uint32_t it = 0;
  for (int t = first; t < count; t += stride) {
    int b, I, J, h;
    unpack_tile(a.tiles[t], b, I, J, h);
    if (!load_params(a, b).active) continue;
    if (!finish_entry(a, it, sh, abort_flag, lane, lim)) return;
    ++it;
  }
}

// The finisher warp of a CTA-pair kernel: the CTA's tiles are
// 2 (uw u + k) + rank for its units u = cl, cl + ncl, ... < nunits and
// k < uw (uw super tiles per unit), in the epilogue warps' order.
__device__ __forceinline__ void finisher_pair(const SqArgs& a, int cl, int ncl, int nunits, int uw, int rank,
                                              Shared& sh, volatile int* abort_flag, int lane) {
  using namespace sp2::tc;
  const unsigned long long lim = wait_limit(a);
  uint32_t it = 0;
  for (int u = cl; u < nunits; u += ncl) {
    for (int k = 0; k < uw; ++k) {
      const int t = 2 * (uw * u + k) + rank;
      int b, I, J, h;
      unpack_tile(a.tiles[t], b, I, J, h);
      if (!load_params(a, b).active) continue;
      if (!finish_entry(a, it, sh, abort_flag, lane, lim)) return;
      ++it;
    }
  }
}

}  // namespace epi
}  // namespace sp2
