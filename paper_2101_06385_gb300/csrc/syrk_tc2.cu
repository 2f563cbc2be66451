// Single-accumulator split-FP16 squaring on tcgen05 with a double-buffered
// TMEM accumulator, run by CTA pairs that share the B operand through TMA
// multicast (sm_103a).
//
// The two 128-row halves (h = 0, 1) of an upper 256 x 256 super tile need the
// same 256 B rows.  A cluster of two CTAs takes both halves of one super tile;
// each CTA loads its own 128 A rows and one 128-row half of B, and the B half
// is multicast into both CTAs' shared memory, so B is read from L2 once per
// super tile instead of twice.  A stage may be refilled only when both CTAs'
// MMAs have released it (the release is a multicast commit).
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
// CTA = 10 warps, persistent over the upper-tile list (one CTA per SM):
//   warp 0      TMA producer (one thread): hp, lo' of the 128 A rows and of
//               the 256 B rows per 64-wide K stage (96 KB, 2 stages)
//   warp 1      TMEM allocation + MMA issuer (one thread)
//   warps 2..9  epilogue: TMEM lane quarter (warp % 4) x column half
// Plain FP16 (split = false): hi hi only, 48 KB stages, 4 stages.
// Every mbarrier wait is bounded; see syrk_tc.cu for the time-out path.
//
// Operand reads use only the upper super tiles of the planes: a 64-wide K
// block that lies left of the diagonal (super column k < I for the A rows of
// super row I, k < J for B) is read from the stored block (k, I) or (k, J)
// transposed: two 64 x 64 TMA boxes per operand half and an MN-major shared-
// memory descriptor, with the operand's major bit set in the instruction
// descriptor for that K block.  So the planes need only be written for the
// upper super tiles (SqArgs::tri_planes).
#include <cuda.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"
#include "epilogue.cuh"

namespace sp2 {
namespace tc2 {

using namespace sp2::tc;

constexpr int STAGE_SPLIT = 2 * A_BYTES + 2 * B_BYTES;  // 96 KB: hpA loA hpB loB
constexpr int STAGE_PLAIN = A_BYTES + B_BYTES;          // 48 KB: hiA hiB
constexpr int STAGES_SPLIT = 2;
constexpr int STAGES_PLAIN = 4;
constexpr int EPI_WARPS = epi::WARPS;
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr uint32_t TMEM_COLS = 512;  // two 256-column accumulators

// one 64 x 64 FP16 box of a transposed read
constexpr int T_BOX = 64 * 64 * 2;
// stage offsets (split): hpA, loA (A_BYTES each), hpB, loB (B_BYTES each)
constexpr int OFF_HPA = 0, OFF_LOA = A_BYTES, OFF_HPB = 2 * A_BYTES, OFF_LOB = 2 * A_BYTES + B_BYTES;

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive;\n\tbarrier.cluster.wait;" ::: "memory");
}

// TMA load multicast to the CTAs in mask: same shared offset in each, each
// destination CTA's mbarrier at that offset receives the byte count.
__device__ __forceinline__ void tma_load_3d_mc(void* dst, const CUtensorMap* tm, int c0, int c1, int c2, uint64_t* bar,
                                               uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.multicast::cluster "
      "[%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar)), "h"(mask)
      : "memory");
}

// Arrive on the mbarrier at this offset in every CTA of mask once all prior
// tcgen05 operations of this thread have completed.
__device__ __forceinline__ void mma_commit_mc(uint64_t* bar, uint16_t mask) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
                   smem_u32(bar)),
               "h"(mask)
               : "memory");
}

// RO: readout mode of the epilogue (finite-temperature expansion).
// tm_p0T / tm_p1T: the planes with 64 x 64 boxes (transposed reads).
template <bool SPLIT, bool RO>
__global__ void __launch_bounds__(THREADS, 1)
    syrk_tc2_kernel(const __grid_constant__ CUtensorMap tm_p0A, const __grid_constant__ CUtensorMap tm_p1A,
                    const __grid_constant__ CUtensorMap tm_p0B, const __grid_constant__ CUtensorMap tm_p1B,
                    const __grid_constant__ CUtensorMap tm_p0T, const __grid_constant__ CUtensorMap tm_p1T,
                    const SqArgs a) {
  constexpr int STAGES = SPLIT ? STAGES_SPLIT : STAGES_PLAIN;
  constexpr int STAGE_BYTES = SPLIT ? STAGE_SPLIT : STAGE_PLAIN;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tmem_full = empty + STAGES;   // [2]
  uint64_t* tmem_empty = tmem_full + 2;   // [2]
  uint64_t* drain = tmem_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  __shared__ int s_abort;
  __shared__ epi::Shared s_epi;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    s_abort = 0;
    epi::init(s_epi);
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 2);  // released by both CTAs' MMAs
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tmem_full[i], 1);
      mbar_init(&tmem_empty[i], EPI_WARPS);
    }
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
  // the peer's barriers must exist before any multicast reaches them
  cluster_sync();
  const uint32_t tmem_base = *tmem_slot;
  volatile int* abort_flag = &s_abort;
  const int rank = (int)cluster_rank();
  const int cl = blockIdx.x >> 1, ncl = gridDim.x >> 1;
  const int nsuper = a.ntiles >> 1;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      uint32_t armed[STAGES];
#pragma unroll
      for (int s = 0; s < STAGES; ++s) armed[s] = 0;
      for (int u = cl; u < nsuper && ok; u += ncl) {
        const int t = 2 * u + rank;
        int b, I, J, h;
        unpack_tile(a.tiles[t], b, I, J, h);
        if (!load_params(a, b).active) continue;
        const int N = a.Ns[b];
        const int rowA = I * BN + h * BM, rowB = J * BN + rank * BM;
        const int nk = (N + BK - 1) / BK;
        for (int kb = 0; kb < nk; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag)) {
            ok = false;
            break;
          }
          uint8_t* st = smem + stage * STAGE_BYTES;
          mbar_expect_tx(&full[stage], STAGE_BYTES);
          const int k0 = kb * BK;
          const int ks = k0 / BN;  // super column of this K block
          // A rows: K-major from (I, k) on or right of the diagonal, else
          // the stored (k, I) transposed as two 64 x 64 boxes
          uint8_t* a0 = st + (SPLIT ? OFF_HPA : 0);
          if (ks >= I) {
            tma_load_3d(a0, &tm_p0A, k0, rowA, b, &full[stage]);
            if (SPLIT) tma_load_3d(st + OFF_LOA, &tm_p1A, k0, rowA, b, &full[stage]);
          } else {
            tma_load_3d(a0, &tm_p0T, rowA, k0, b, &full[stage]);
            tma_load_3d(a0 + T_BOX, &tm_p0T, rowA + 64, k0, b, &full[stage]);
            if (SPLIT) {
              tma_load_3d(st + OFF_LOA, &tm_p1T, rowA, k0, b, &full[stage]);
              tma_load_3d(st + OFF_LOA + T_BOX, &tm_p1T, rowA + 64, k0, b, &full[stage]);
            }
          }
          // this CTA's half of the B rows, multicast into both CTAs
          uint8_t* b0 = st + (SPLIT ? OFF_HPB : A_BYTES) + rank * (B_BYTES / 2);
          if (ks >= J) {
            tma_load_3d_mc(b0, &tm_p0B, k0, rowB, b, &full[stage], 0x3);
            if (SPLIT)
              tma_load_3d_mc(st + OFF_LOB + rank * (B_BYTES / 2), &tm_p1B, k0, rowB, b, &full[stage], 0x3);
          } else {
            tma_load_3d_mc(b0, &tm_p0T, rowB, k0, b, &full[stage], 0x3);
            tma_load_3d_mc(b0 + T_BOX, &tm_p0T, rowB + 64, k0, b, &full[stage], 0x3);
            if (SPLIT) {
              uint8_t* b1 = st + OFF_LOB + rank * (B_BYTES / 2);
              tma_load_3d_mc(b1, &tm_p1T, rowB, k0, b, &full[stage], 0x3);
              tma_load_3d_mc(b1 + T_BOX, &tm_p1T, rowB + 64, k0, b, &full[stage], 0x3);
            }
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
          while (!mbar_try_wait(&full[s], (armed[s] - 1u) & 1u) && globaltimer() - t0 < kTimeoutNs) {
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
      for (int u = cl; u < nsuper && ok; u += ncl) {
        const int t = 2 * u + rank;
        int b, I, J, h;
        unpack_tile(a.tiles[t], b, I, J, h);
        if (!load_params(a, b).active) continue;
        const int N = a.Ns[b];
        const int nk = (N + BK - 1) / BK;
        const uint32_t buf = it & 1u;
        (void)h;
        // the k-th use of a buffer waits for the epilogue's (k-1)-th release
        if (!mbar_wait(&tmem_empty[buf], ((it >> 1) & 1u) ^ 1u, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem_base + buf * BN;
        for (int kb = 0; kb < nk; ++kb) {
          if (!mbar_wait(&full[stage], phase, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = smem_u32(smem + stage * STAGE_BYTES);
          // operands left of the diagonal arrived transposed (MN-major)
          const int sc = kb * BK / BN;
          const bool ta = sc < I, tb = sc < J;
          const uint32_t idesc = IDESC | (ta ? IDESC_A_MN : 0u) | (tb ? IDESC_B_MN : 0u);
#pragma unroll
          for (int ks = 0; ks < BK / UMMA_K; ++ks) {
            // K step ks: 32 B along a K-major row, or two 8-row K groups
            const uint32_t oa = ta ? ks * 2048u : ks * UMMA_K * 2u;
            const uint32_t ob = tb ? ks * 2048u : ks * UMMA_K * 2u;
            const uint32_t acc = (kb > 0 || ks > 0) ? 1u : 0u;
            if (SPLIT) {
              const uint64_t dhpA = ta ? make_desc_mn128(st + OFF_HPA + oa) : make_desc_sw128(st + OFF_HPA + oa);
              const uint64_t dloA = ta ? make_desc_mn128(st + OFF_LOA + oa) : make_desc_sw128(st + OFF_LOA + oa);
              const uint64_t dhpB = tb ? make_desc_mn128(st + OFF_HPB + ob) : make_desc_sw128(st + OFF_HPB + ob);
              const uint64_t dloB = tb ? make_desc_mn128(st + OFF_LOB + ob) : make_desc_sw128(st + OFF_LOB + ob);
              mma_f16_id(d, dhpA, dhpB, idesc, acc);  // hp hp
              mma_f16_id(d, dloA, dhpB, idesc, 1u);   // lo' hp
              mma_f16_id(d, dhpA, dloB, idesc, 1u);   // hp lo'
            } else {
              const uint64_t dA = ta ? make_desc_mn128(st + oa) : make_desc_sw128(st + oa);
              const uint64_t dB = tb ? make_desc_mn128(st + A_BYTES + ob) : make_desc_sw128(st + A_BYTES + ob);
              mma_f16_id(d, dA, dB, idesc, acc);
            }
          }
          mma_commit_mc(&empty[stage], 0x3);  // release the stage in both CTAs
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
        while (!mbar_try_wait(drain, 0) && globaltimer() - t0 < kTimeoutNs) {
        }
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int ew = warp - 2;  // 0..7
    const int q = warp & 3;   // TMEM lane quarter
    uint32_t it = 0;
    for (int u = cl; u < nsuper; u += ncl) {
      const int t = 2 * u + rank;
      const int rc = epi::tile<SPLIT, false, RO>(a, t, it, tmem_base, tmem_full, tmem_empty, abort_flag, s_epi, ew, q,
                                                  lane);
      if (rc < 0) break;
      it += (uint32_t)rc;
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // no CTA leaves while its peer may still multicast into it or arrive on it
  cluster_sync();
  if (warp == 1) {
    __syncwarp();
    tmem_dealloc(tmem_base, TMEM_COLS);
  }
}

}  // namespace tc2

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

size_t syrk_tc2_smem_bytes(bool split) {
  const int stages = split ? tc2::STAGES_SPLIT : tc2::STAGES_PLAIN;
  const int sb = split ? tc2::STAGE_SPLIT : tc2::STAGE_PLAIN;
  return (size_t)stages * sb + 1024 /* alignment slack */ + 256 /* barriers */;
}

cudaError_t launch_syrk_tc2(const SqArgs& a, const CUtensorMap* tm, bool split, int grid, cudaStream_t st) {
  // grid: number of CTAs, even (two per cluster); a.ntiles = 2 x super tiles
  const size_t smem = syrk_tc2_smem_bytes(split);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(grid & ~1), 1, 1);
  cfg.blockDim = dim3(tc2::THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e;
  if (a.R) {
    if (split) {
      e = set_smem_once(tc2::syrk_tc2_kernel<true, true>, (int)smem, 3);
      if (e != cudaSuccess) return e;
      e = cudaLaunchKernelEx(&cfg, tc2::syrk_tc2_kernel<true, true>, tm[0], tm[1], tm[2], tm[3], tm[4], tm[5], a);
    } else {
      e = set_smem_once(tc2::syrk_tc2_kernel<false, true>, (int)smem, 2);
      if (e != cudaSuccess) return e;
      e = cudaLaunchKernelEx(&cfg, tc2::syrk_tc2_kernel<false, true>, tm[0], tm[1], tm[2], tm[3], tm[4], tm[5], a);
    }
  } else if (split) {
    e = set_smem_once(tc2::syrk_tc2_kernel<true, false>, (int)smem, 1);
    if (e != cudaSuccess) return e;
    e = cudaLaunchKernelEx(&cfg, tc2::syrk_tc2_kernel<true, false>, tm[0], tm[1], tm[2], tm[3], tm[4], tm[5], a);
  } else {
    e = set_smem_once(tc2::syrk_tc2_kernel<false, false>, (int)smem, 0);
    if (e != cudaSuccess) return e;
    e = cudaLaunchKernelEx(&cfg, tc2::syrk_tc2_kernel<false, false>, tm[0], tm[1], tm[2], tm[3], tm[4], tm[5], a);
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace sp2
