// Split-FP16 symmetric squaring on the 5th-generation tensor cores (sm_103a):
// tcgen05.mma with FP32 accumulators in tensor memory, operands staged in
// shared memory by TMA, fused SP2 layer epilogue.
//
// The two-accumulator kernel on hi/lo planes; it serves the allocation-free
// solve (noalloc.cu).  The other solves use the single-accumulator kernels
// of syrk_tc1.cu / syrk_tc2.cu.
//
// Alg. 2 / Eq. 14: with Y ~ hi + 2^-s lo (Eq. 12, lo scaled by 2^s),
//     P = Y^2 ~ hi hi + 2^-s (lo hi + hi lo)          (the lo lo term is dropped)
// Y is symmetric, so tile (I, J) of P is  sum_k Y[I, k] Y[J, k]^T: both MMA
// operands are row panels in K-major layout.  Only the upper 256 x 256 super
// tiles (I <= J) are computed (the symmetric-half remark under Eq. 14); each
// is two 128 x 256 CTA tiles.  Off-diagonal super tiles are stored twice
// (mirrored) so every layer again reads full row panels.
//
// CTA = 6 warps, persistent over a static tile list:
//   warp 0      TMA producer (one thread): hi/lo of rows I (128) and J (256)
//   warp 1      TMEM allocation + MMA issuer (one thread)
//   warps 2..5  epilogue: TMEM -> registers, Y' = ca Y + cb P + cc I,
//               re-split to hi/lo, mirrored stores, FP64 trace partials
// TMEM: ACC0 = hi hi in columns [0, 256), ACC1 = lo hi + hi lo in [256, 512).
// Every mbarrier wait is bounded (globaltimer); on time-out the CTA records
// SP2_ERR_DEVICE_TIMEOUT, stops issuing, drains and frees its TMEM.
#include <cuda.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"
#include "tile_finish.cuh"

namespace sp2 {

namespace tc {

constexpr int STAGE_SPLIT = 2 * A_BYTES + 2 * B_BYTES;  // 96 KB: hiA loA hiB loB
constexpr int STAGE_PLAIN = A_BYTES + B_BYTES;          // 48 KB: hiA hiB
constexpr int STAGES_SPLIT = 2;
constexpr int STAGES_PLAIN = 4;
constexpr int THREADS = 192;

template <bool SPLIT>
__global__ void __launch_bounds__(THREADS, 1)
    syrk_tc_kernel(const __grid_constant__ CUtensorMap tm_hiA, const __grid_constant__ CUtensorMap tm_loA,
                   const __grid_constant__ CUtensorMap tm_hiB, const __grid_constant__ CUtensorMap tm_loB,
                   const __grid_constant__ CUtensorMap tm_hiA2, const __grid_constant__ CUtensorMap tm_loA2,
                   const __grid_constant__ CUtensorMap tm_hiB2, const __grid_constant__ CUtensorMap tm_loB2,
                   const SqArgs a) {
  constexpr int STAGES = SPLIT ? STAGES_SPLIT : STAGES_PLAIN;
  constexpr int STAGE_BYTES = SPLIT ? STAGE_SPLIT : STAGE_PLAIN;
  constexpr uint32_t TMEM_COLS = SPLIT ? 512 : 256;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tmem_full = empty + STAGES;
  uint64_t* tmem_empty = tmem_full + 1;
  uint64_t* drain = tmem_empty + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  __shared__ int s_abort;
  __shared__ double s_red[4][5];
  __shared__ int s_got[4];

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(tmem_full, 1);
    mbar_init(tmem_empty, 4);
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  volatile int* abort_flag = &s_abort;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      uint32_t armed[STAGES];
#pragma unroll
      for (int s = 0; s < STAGES; ++s) armed[s] = 0;
      for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
        int b, I, J, h;
        unpack_tile(a.tiles[t], b, I, J, h);
        if (!load_params(a, b).active) continue;
        const int N = a.Ns[b];
        const int rowA = I * BN + h * BM, rowB = J * BN;
        const int nk = (N + BK - 1) / BK;
        const int nseg = a.nseg > 1 ? 2 : 1;
        for (int kb = 0; kb < nk * nseg; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag)) {
            ok = false;
            break;
          }
          uint8_t* st = smem + stage * STAGE_BYTES;
          mbar_expect_tx(&full[stage], STAGE_BYTES);
          // second K segment (two-operand product A B^T + B A^T): swap the maps
          const bool seg2 = kb >= nk;
          const int k0 = (seg2 ? kb - nk : kb) * BK;
          const CUtensorMap* mhA = seg2 ? &tm_hiA2 : &tm_hiA;
          const CUtensorMap* mlA = seg2 ? &tm_loA2 : &tm_loA;
          const CUtensorMap* mhB = seg2 ? &tm_hiB2 : &tm_hiB;
          const CUtensorMap* mlB = seg2 ? &tm_loB2 : &tm_loB;
          if (SPLIT) {
            tma_load_3d(st, mhA, k0, rowA, b, &full[stage]);
            tma_load_3d(st + A_BYTES, mlA, k0, rowA, b, &full[stage]);
            tma_load_3d(st + 2 * A_BYTES, mhB, k0, rowB, b, &full[stage]);
            tma_load_3d(st + 2 * A_BYTES + B_BYTES, mlB, k0, rowB, b, &full[stage]);
          } else {
            tma_load_3d(st, mhA, k0, rowA, b, &full[stage]);
            tma_load_3d(st + A_BYTES, mhB, k0, rowB, b, &full[stage]);
          }
          ++armed[stage];
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok || *abort_flag) {
        atomicExch(a.err, (int)SP2_ERR_DEVICE_TIMEOUT);
        // Drain: the copies this thread issued land before the CTA exits
        // (the k-th arming of a stage completes the phase of parity (k-1)&1).
        for (int s = 0; s < STAGES; ++s) {
          if (armed[s] == 0) continue;
          const uint64_t t0 = globaltimer();
          while (!mbar_try_wait(&full[s], (armed[s] - 1u) & 1u) && globaltimer() - t0 < kTimeoutNs) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, acc_phase = 0;
      bool ok = true;
      bool issued = false;
      for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
        int b, I, J, h;
        unpack_tile(a.tiles[t], b, I, J, h);
        if (!load_params(a, b).active) continue;
        const int N = a.Ns[b];
        const int nk = (N + BK - 1) / BK;
        if (!mbar_wait(tmem_empty, acc_phase ^ 1u, abort_flag)) {
          ok = false;
          break;
        }
        acc_phase ^= 1u;
        tc_fence_after();
        const int nseg = a.nseg > 1 ? 2 : 1;
        for (int kb = 0; kb < nk * nseg; ++kb) {
          if (!mbar_wait(&full[stage], phase, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = smem_u32(smem + stage * STAGE_BYTES);
#pragma unroll
          for (int ks = 0; ks < BK / UMMA_K; ++ks) {
            const uint32_t koff = ks * UMMA_K * 2;  // bytes within the 128-byte row
            const uint32_t acc = (kb > 0 || ks > 0) ? 1u : 0u;
            if (SPLIT) {
              const uint64_t dhiA = make_desc_sw128(st + koff);
              const uint64_t dloA = make_desc_sw128(st + A_BYTES + koff);
              const uint64_t dhiB = make_desc_sw128(st + 2 * A_BYTES + koff);
              const uint64_t dloB = make_desc_sw128(st + 2 * A_BYTES + B_BYTES + koff);
              mma_f16(tmem_base, dhiA, dhiB, acc);              // ACC0 += hi_I hi_J^T
              mma_f16(tmem_base + BN, dloA, dhiB, acc);         // ACC1 += lo_I hi_J^T
              mma_f16(tmem_base + BN, dhiA, dloB, 1u);          // ACC1 += hi_I lo_J^T
            } else {
              const uint64_t dhiA = make_desc_sw128(st + koff);
              const uint64_t dhiB = make_desc_sw128(st + A_BYTES + koff);
              mma_f16(tmem_base, dhiA, dhiB, acc);
            }
          }
          mma_commit(&empty[stage]);
          issued = true;
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        mma_commit(tmem_full);
      }
      if (!ok) atomicExch(a.err, (int)SP2_ERR_DEVICE_TIMEOUT);
      if (issued) {
        // all MMAs of this CTA have completed once this commit lands
        mma_commit(drain);
        const uint64_t t0 = globaltimer();
        while (!mbar_try_wait(drain, 0) && globaltimer() - t0 < kTimeoutNs) {
        }
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;                 // TMEM lane quarter of this warp
    const int row_local = q * 32 + lane;
    uint32_t acc_phase = 0;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
      int b, I, J, h;
      unpack_tile(a.tiles[t], b, I, J, h);
      const LayerParams p = load_params(a, b);
      if (!p.active) continue;
      const int N = a.Ns[b];
      const int r = I * BN + h * BM + row_local;
      const int cb0 = J * BN;
      const bool mirror = (I != J);
      const bool outD = (p.out_mode == OUT_D);
      // FP64 row norm for the diagonal, fetched before the accumulator wait
      const double rn_r = (!mirror && a.rn && r < N) ? a.rn[(long long)b * a.ld_rn + r] : 0.0;
      const bool got = mbar_wait(tmem_full, acc_phase, abort_flag);
      // the four epilogue warps take one decision: go on only if all of them
      // saw the accumulator arrive (s_got is rewritten only after the
      // end-of-tile barriers below)
      if (lane == 0) s_got[q] = got ? 1 : 0;
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (!(s_got[0] & s_got[1] & s_got[2] & s_got[3])) {
        if (!got && lane == 0) atomicExch(a.err, (int)SP2_ERR_DEVICE_TIMEOUT);
        break;
      }
      acc_phase ^= 1u;
      tc_fence_after();

      float* Y = a.Yout + (long long)b * a.slot_y;
      const float* Yold = a.Yin + (long long)b * a.slot_y;
      const long long ld = a.ld_y;
      __half* ho = a.hi_out ? a.hi_out + (long long)b * a.slot_h : nullptr;
      __half* lo_ = a.lo_out ? a.lo_out + (long long)b * a.slot_h : nullptr;
      const long long ldh = a.ld_h;
      float* D = outD ? a.Dptr[b] : nullptr;
      double tr = 0.0, sq = 0.0;
      double dtr = 0.0, dgy = 0.0, dpy = 0.0;  // adjoint-mode dot products
      const uint32_t lane_base = (uint32_t)(q * 32) << 16;

      for (int ch = 0; ch < BN / 32; ++ch) {
        uint32_t v0[32], v1[32];
        __syncwarp();
        tmem_ld32(tmem_base + lane_base + ch * 32, v0);
        if (SPLIT) tmem_ld32(tmem_base + lane_base + BN + ch * 32, v1);
        tmem_ld_wait();
        const int c0 = cb0 + ch * 32;
        float y[32];
        float sqf = 0.f;
        float ydiag = 0.f;
        if (r < N) {
          const bool full_chunk = (c0 + 32 <= N) && ((ld & 3) == 0);
          if (full_chunk) {
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
          // the diagonal element of row r, if it lies in this chunk (I == J only)
          const int jd = r - c0;
          const bool dchunk = !mirror && (unsigned)jd < 32u;
          float yold_d = 0.f, p_d = 0.f;
          if (dchunk) {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (j == jd) {
                yold_d = y[j];
                p_d = SPLIT ? fmaf(__uint_as_float(v1[j]), a.lo_unscale, __uint_as_float(v0[j])) : __uint_as_float(v0[j]);
              }
          }
          if (a.aux) {
            // adjoint mode: tr Yin, <Yin, aux>, <P, aux> on the old values
            const float* ax = a.aux + (long long)b * a.slot_y + (long long)r * ld + c0;
            float gy = 0.f, py = 0.f;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              if (c0 + j < N) {
                const float xv = ax[j];
                const float P = SPLIT ? fmaf(__uint_as_float(v1[j]), a.lo_unscale, __uint_as_float(v0[j])) : __uint_as_float(v0[j]);
                gy = fmaf(y[j], xv, gy);
                py = fmaf(P, xv, py);
              }
            }
            if (dchunk) dtr += (double)yold_d;
            dgy += (double)gy;
            dpy += (double)py;
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float P = SPLIT ? fmaf(__uint_as_float(v1[j]), a.lo_unscale, __uint_as_float(v0[j])) : __uint_as_float(v0[j]);
            const float yn = fmaf(p.ca, y[j], p.cb * P);
            y[j] = (c0 + j < N) ? yn : 0.f;
          }
          if (dchunk) {
            // diagonal of Y^2 from the FP64 row norms (unbiased), update in
            // FP64, once per row outside the unrolled element loop
            const double pd = a.rn ? rn_r : (double)p_d;
            const double yd = p.ca_d * (double)yold_d + p.cb_d * pd + p.cc_d;
            tr += yd;
            const float ydf = (float)yd;
            if (outD) ydiag = (float)(yd + p.alpha_out);
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (j == jd) y[j] = ydf;
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) sqf = fmaf(y[j], y[j], sqf);
          sq += (double)sqf;
          if (outD) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int c = c0 + j;
              if (c < N) D[(long long)r * N + c] = (r == c) ? ydiag : y[j];
            }
          } else {
            if (full_chunk) {
              float4* dst = reinterpret_cast<float4*>(Y + (long long)r * ld + c0);
#pragma unroll
              for (int j4 = 0; j4 < 8; ++j4)
                dst[j4] = make_float4(y[4 * j4], y[4 * j4 + 1], y[4 * j4 + 2], y[4 * j4 + 3]);
            } else {
#pragma unroll
              for (int j = 0; j < 32; ++j)
                if (c0 + j < N) Y[(long long)r * ld + c0 + j] = y[j];
            }
            if (ho) {
              // 32 halves = 64 B per part; the padded row tail [N, ld_h) stays zero
              __align__(16) __half hh[32], ll[32];
#pragma unroll
              for (int j = 0; j < 32; ++j) split_fp16(y[j], a.lo_scale, hh[j], ll[j]);
              // columns >= N hold y = 0, so the padded row tail [N, ld_h) stays zero
              if (c0 + 32 <= (int)ldh) {
                uint4* dh = reinterpret_cast<uint4*>(ho + (long long)r * ldh + c0);
                const uint4* sh = reinterpret_cast<const uint4*>(hh);
#pragma unroll
                for (int j4 = 0; j4 < 4; ++j4) dh[j4] = sh[j4];
                if (lo_) {
                  uint4* dl = reinterpret_cast<uint4*>(lo_ + (long long)r * ldh + c0);
                  const uint4* sl = reinterpret_cast<const uint4*>(ll);
#pragma unroll
                  for (int j4 = 0; j4 < 4; ++j4) dl[j4] = sl[j4];
                }
              } else {
                for (int j = 0; j < 32; ++j)
                  if (c0 + j < (int)ldh) {
                    ho[(long long)r * ldh + c0 + j] = hh[j];
                    if (lo_) lo_[(long long)r * ldh + c0 + j] = ll[j];
                  }
              }
            }
          }
        }
        // mirrored store: lanes hold consecutive rows r -> consecutive columns
        if (mirror) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int c = c0 + j;
            if (c < N && r < N) {
              if (outD) {
                D[(long long)c * N + r] = y[j];
              } else {
                Y[(long long)c * ld + r] = y[j];
                if (ho) {
                  __half hh, ll;
                  split_fp16(y[j], a.lo_scale, hh, ll);
                  ho[(long long)c * ldh + r] = hh;
                  if (lo_) lo_[(long long)c * ldh + r] = ll;
                }
              }
            }
          }
        }
      }
      // accumulator drained: let the MMA warp start the next tile
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tmem_empty);

      if (mirror) {
        sq *= 2.0;
        dgy *= 2.0;
        dpy *= 2.0;
      }
      tr = warp_sum_d(tr);
      sq = warp_sum_d(sq);
      if (a.aux) {
        dtr = warp_sum_d(dtr);
        dgy = warp_sum_d(dgy);
        dpy = warp_sum_d(dpy);
      }
      if (lane == 0) {
        s_red[q][0] = tr;
        s_red[q][1] = sq;
        s_red[q][2] = dtr;
        s_red[q][3] = dgy;
        s_red[q][4] = dpy;
      }
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (warp == 2) {
        double T = 0.0, Q = 0.0;
        if (lane == 0) {
          double d0 = 0.0, d1 = 0.0, d2 = 0.0;
          for (int k = 0; k < 4; ++k) {
            T += s_red[k][0];
            Q += s_red[k][1];
            d0 += s_red[k][2];
            d1 += s_red[k][3];
            d2 += s_red[k][4];
          }
          if (a.aux) {
            a.tile_dots[3 * (long long)t + 0] = d0;
            a.tile_dots[3 * (long long)t + 1] = d1;
            a.tile_dots[3 * (long long)t + 2] = d2;
          }
        }
        finish_tile_warp(a, t, b, T, Q, p.out_mode);
      }
      asm volatile("bar.sync 1, 128;" ::: "memory");
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    __syncwarp();
    tmem_dealloc(tmem_base, TMEM_COLS);
  }
}

}  // namespace tc

size_t syrk_tc_smem_bytes(bool split) {
  const int stages = split ? tc::STAGES_SPLIT : tc::STAGES_PLAIN;
  const int sb = split ? tc::STAGE_SPLIT : tc::STAGE_PLAIN;
  return (size_t)stages * sb + 1024 /* alignment slack */ + 256 /* barriers */;
}

cudaError_t launch_syrk_tc(const SqArgs& a, const CUtensorMap* tm, bool split, int grid, cudaStream_t st) {
  // one K segment uses tm[0..3]; two segments also tm[4..7]
  const CUtensorMap* t2 = (a.nseg == 2) ? tm + 4 : tm;
  const size_t smem = syrk_tc_smem_bytes(split);
  cudaError_t e;
  if (split) {
    e = cudaFuncSetAttribute(tc::syrk_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    tc::syrk_tc_kernel<true><<<grid, tc::THREADS, smem, st>>>(tm[0], tm[1], tm[2], tm[3], t2[0], t2[1], t2[2],
                                                              t2[3], a);
  } else {
    e = cudaFuncSetAttribute(tc::syrk_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    tc::syrk_tc_kernel<false><<<grid, tc::THREADS, smem, st>>>(tm[0], tm[1], tm[2], tm[3], t2[0], t2[1], t2[2],
                                                               t2[3], a);
  }
  return cudaGetLastError();
}

}  // namespace sp2
