// Single-accumulator split-FP16 squaring on tcgen05 with a double-buffered
// TMEM accumulator (sm_103a).
//
// Alg. 2 / Eq. 14 with both parts scaled by 2^s (Eq. 12: hi = fp16(Y),
// lo' = fp16(2^s (Y - hi)); hp = 2^s hi is exact in FP16 for |Y| < 2^(15-s)):
//     2^(2s) P = hp hp + lo' hp + hp lo',
// so only two FP16 planes (hp, lo') are stored and loaded, and the three
// products accumulate into ONE FP32 TMEM accumulator of 128 x 256 (256
// columns).  Scaling by powers of two commutes with every rounding, so the
// result equals that of the unscaled products hi hi + lo hi + hi lo.  Two such accumulators fit in the 512 TMEM
// columns: while the epilogue warps drain tile t from one, the MMA issuer
// fills the other with tile t+1, and the epilogue (FP32 update, re-split,
// row and mirrored stores, traces) runs under the next tile's MMAs.
//
// CTA = 11 warps, persistent over the upper-tile list (one CTA per SM):
//   warp 0      TMA producer (one thread): hp, lo' of the 128 A rows and of
//               the 256 B rows per 64-wide K stage (96 KB, 2 stages)
//   warp 1      TMEM allocation + MMA issuer (one thread)
//   warps 2..9  epilogue: TMEM lane quarter (warp % 4) x column half
//   warp 10     finisher: publishes each tile's sums, runs the control steps
// Plain FP16 (split = false): hi hi only, 48 KB stages, 4 stages.
// Every mbarrier wait is bounded; see syrk_tc.cu for the time-out path.
#include <cuda.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"
#include "epilogue.cuh"

namespace sp2 {
namespace tc1 {

using namespace sp2::tc;

constexpr int STAGE_SPLIT = 2 * A_BYTES + 2 * B_BYTES;  // 96 KB: hpA loA hpB loB
constexpr int STAGE_PLAIN = A_BYTES + B_BYTES;          // 48 KB: hiA hiB
constexpr int STAGES_SPLIT = 2;
constexpr int STAGES_PLAIN = 4;
constexpr int EPI_WARPS = epi::WARPS;
constexpr int FIN_WARP = 2 + EPI_WARPS;  // the finisher warp (after the epilogue warps)
constexpr int THREADS = 64 + 32 * EPI_WARPS + 32;
constexpr uint32_t TMEM_COLS = 512;  // two 256-column accumulators

// stage offsets (split): hpA, loA (A_BYTES each), hpB, loB (B_BYTES each)
constexpr int OFF_HPA = 0, OFF_LOA = A_BYTES, OFF_HPB = 2 * A_BYTES, OFF_LOB = 2 * A_BYTES + B_BYTES;

// NSEG2: P = A_1 B_1^T + A_2 B_2^T over two K segments (the second map set
// holds the second segment's operands) with the adjoint-mode epilogue: the
// split SYR2K Y G + G Y of the network adjoint.
template <bool SPLIT, bool NSEG2>

__global__ void __launch_bounds__(THREADS, 1)
    syrk_tc1_kernel(const __grid_constant__ CUtensorMap tm_p0A, const __grid_constant__ CUtensorMap tm_p1A,
                    const __grid_constant__ CUtensorMap tm_p0B, const __grid_constant__ CUtensorMap tm_p1B,
                    const __grid_constant__ CUtensorMap tm2_p0A, const __grid_constant__ CUtensorMap tm2_p1A,
                    const __grid_constant__ CUtensorMap tm2_p0B, const __grid_constant__ CUtensorMap tm2_p1B,
                    const SqArgs a) {
  constexpr int NSEG = NSEG2 ? 2 : 1;
  constexpr int STAGES = SPLIT ? STAGES_SPLIT : STAGES_PLAIN;
  constexpr int STAGE_BYTES = SPLIT ? STAGE_SPLIT : STAGE_PLAIN;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tmem_full = empty + STAGES;   // [2]
  uint64_t* tmem_empty = tmem_full + 2;   // [2]
  uint64_t* drain = tmem_empty + 2;
  uint64_t* never = drain + 1;  // fault injection: nothing arrives on it
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(never + 1);
  // the epilogue warps' staging buffers, after the 256 bytes of barriers
  float* trbuf = reinterpret_cast<float*>(smem + STAGES * STAGE_BYTES + 256);
  __shared__ int s_abort;
  __shared__ epi::Shared s_epi;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    s_abort = 0;
    epi::init(s_epi);
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tmem_full[i], 1);
      mbar_init(&tmem_empty[i], EPI_WARPS);
    }
    mbar_init(drain, 1);
    mbar_init(never, 1);
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
  const unsigned long long lim = wait_limit(a);

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
        for (int kb = 0; kb < nk * NSEG; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, lim)) {
            ok = false;
            break;
          }
          uint8_t* st = smem + stage * STAGE_BYTES;
          mbar_expect_tx(&full[stage], STAGE_BYTES);
          const bool seg2 = NSEG2 && kb >= nk;
          const int k0 = (seg2 ? kb - nk : kb) * BK;
          const CUtensorMap* m0A = seg2 ? &tm2_p0A : &tm_p0A;
          const CUtensorMap* m0B = seg2 ? &tm2_p0B : &tm_p0B;
          if (SPLIT) {
            tma_load_3d(st + OFF_HPA, m0A, k0, rowA, b, &full[stage]);
            tma_load_3d(st + OFF_LOA, seg2 ? &tm2_p1A : &tm_p1A, k0, rowA, b, &full[stage]);
            tma_load_3d(st + OFF_HPB, m0B, k0, rowB, b, &full[stage]);
            tma_load_3d(st + OFF_LOB, seg2 ? &tm2_p1B : &tm_p1B, k0, rowB, b, &full[stage]);
          } else {
            tma_load_3d(st, m0A, k0, rowA, b, &full[stage]);
            tma_load_3d(st + A_BYTES, m0B, k0, rowB, b, &full[stage]);
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
        for (int s = 0; s < STAGES; ++s) {
          if (armed[s] == 0) continue;
          const uint64_t t0 = globaltimer();
          while (!mbar_try_wait(&full[s], (armed[s] - 1u) & 1u) && globaltimer() - t0 < lim) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, it = 0;
      bool ok = true, issued = false;
      // injected fault (SqArgs::stall): a wait that runs out after lim
      if (a.stall && !mbar_wait(never, 0, abort_flag, lim)) ok = false;
      for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
        int b, I, J, h;
        unpack_tile(a.tiles[t], b, I, J, h);
        if (!load_params(a, b).active) continue;
        const int N = a.Ns[b];
        const int nk = (N + BK - 1) / BK;
        const uint32_t buf = it & 1u;
        // the k-th use of a buffer waits for the epilogue's (k-1)-th release
        if (!mbar_wait(&tmem_empty[buf], ((it >> 1) & 1u) ^ 1u, abort_flag, lim)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem_base + buf * BN;
        for (int kb = 0; kb < nk * NSEG; ++kb) {
          if (!mbar_wait(&full[stage], phase, abort_flag, lim)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = smem_u32(smem + stage * STAGE_BYTES);
#pragma unroll
          for (int ks = 0; ks < BK / UMMA_K; ++ks) {
            const uint32_t koff = ks * UMMA_K * 2;
            const uint32_t acc = (kb > 0 || ks > 0) ? 1u : 0u;
            if (SPLIT) {
              const uint64_t dhpA = make_desc_sw128(st + OFF_HPA + koff);
              const uint64_t dhpB = make_desc_sw128(st + OFF_HPB + koff);
              mma_f16(d, dhpA, dhpB, acc);                                       // hp hp
              mma_f16(d, make_desc_sw128(st + OFF_LOA + koff), dhpB, 1u);        // lo' hp
              mma_f16(d, dhpA, make_desc_sw128(st + OFF_LOB + koff), 1u);        // hp lo'
            } else {
              mma_f16(d, make_desc_sw128(st + koff), make_desc_sw128(st + A_BYTES + koff), acc);
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
        mma_commit(&tmem_full[buf]);
        ++it;
      }
      if (!ok) atomicExch(a.err, (int)SP2_ERR_DEVICE_TIMEOUT);
      if (issued) {
        mma_commit(drain);
        const uint64_t t0 = globaltimer();
        while (!mbar_try_wait(drain, 0) && globaltimer() - t0 < lim) {
        }
      }
    }
  } else if (warp == FIN_WARP) {
    // ------------------------------------------------------------ finisher
    epi::finisher(a, blockIdx.x, gridDim.x, a.ntiles, s_epi, abort_flag, lane);
  } else {
    // ------------------------------------------------------------ epilogue
    const int ew = warp - 2;  // 0..7
    const int q = warp & 3;   // TMEM lane quarter
    uint32_t it = 0;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
      const int rc =
          epi::tile<SPLIT, NSEG2>(a, t, it, tmem_base, tmem_full, tmem_empty, abort_flag, s_epi, ew, q, lane,
                                  trbuf + ew * epi::TR_FLOATS);
      if (rc < 0) break;
      it += (uint32_t)rc;
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

}  // namespace tc1

// The dynamic shared-memory opt-in, once per kernel and device (not a stream
// operation, and kept out of captured launch sequences).
namespace {
template <typename K>
cudaError_t set_smem_once(K kernel, int bytes, int which) {
  static int done_dev[4] = {-1, -1, -1, -1};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (done_dev[which] == dev) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done_dev[which] = dev;
  return e;
}
}  // namespace

size_t syrk_tc1_smem_bytes(bool split) {
  const int stages = split ? tc1::STAGES_SPLIT : tc1::STAGES_PLAIN;
  const int sb = split ? tc1::STAGE_SPLIT : tc1::STAGE_PLAIN;
  return (size_t)stages * sb + 1024 /* alignment slack */ + 256 /* barriers */ + epi::TR_BYTES;
}

cudaError_t launch_syrk_tc1(const SqArgs& a, const CUtensorMap* tm, bool split, int grid, cudaStream_t st) {
  const size_t smem = syrk_tc1_smem_bytes(split);
  // the second map set: segment 2 of the two-segment product, else unused
  const CUtensorMap* t2 = (a.nseg == 2) ? tm + 4 : tm;
  cudaError_t e;
  if (a.nseg == 2) {
    if (split) {
      e = set_smem_once(tc1::syrk_tc1_kernel<true, true>, (int)smem, 2);
      if (e != cudaSuccess) return e;
      tc1::syrk_tc1_kernel<true, true><<<grid, tc1::THREADS, smem, st>>>(tm[0], tm[1], tm[2], tm[3], t2[0], t2[1],
                                                                          t2[2], t2[3], a);
    } else {
      e = set_smem_once(tc1::syrk_tc1_kernel<false, true>, (int)smem, 3);
      if (e != cudaSuccess) return e;
      tc1::syrk_tc1_kernel<false, true><<<grid, tc1::THREADS, smem, st>>>(tm[0], tm[1], tm[2], tm[3], t2[0], t2[1],
                                                                           t2[2], t2[3], a);
    }
  } else if (split) {
    e = set_smem_once(tc1::syrk_tc1_kernel<true, false>, (int)smem, 1);
    if (e != cudaSuccess) return e;
    tc1::syrk_tc1_kernel<true, false><<<grid, tc1::THREADS, smem, st>>>(tm[0], tm[1], tm[2], tm[3], t2[0], t2[1],
                                                                         t2[2], t2[3], a);
  } else {
    e = set_smem_once(tc1::syrk_tc1_kernel<false, false>, (int)smem, 0);
    if (e != cudaSuccess) return e;
    tc1::syrk_tc1_kernel<false, false><<<grid, tc1::THREADS, smem, st>>>(tm[0], tm[1], tm[2], tm[3], t2[0], t2[1],
                                                                          t2[2], t2[3], a);
  }
  return cudaGetLastError();
}

}  // namespace sp2
