// Single-accumulator split-FP16 squaring on tcgen05 run by CTA pairs: one
// M = 256 MMA (tcgen05 .cta_group::2) per K step covers a whole 256 x 256
// upper super tile, with a double-buffered TMEM accumulator (sm_103a).
//
// The two CTAs of a cluster take the two 128-row halves of one super tile
// (I, J).  Each CTA loads, per 64-wide K stage, its own 128 A rows (rows
// I*256 + 128 rank ...) and its own 128 of the 256 B rows (rows J*256 + 128
// rank ...) into its own shared memory with plain TMA loads; the pair MMA,
// issued by one thread of the even CTA, reads the A and B halves of both CTAs
// and writes rows 0-127 of the tile into the even CTA's tensor memory and
// rows 128-255 into the odd CTA's.  So a CTA's stage holds 128 A rows and 128
// B rows (64 KB split, three stages), and the tensor core of each SM reads
// 256 operand rows from shared memory per 128 x 256 x 16 product, against
// 384 for a single-CTA 128 x 256 tile.  Nothing is multicast: the tensor maps
// cover this GPU's own planes and each byte lands only in the CTA that loads
// it.
//
// Synchronisation of a pair:
//   full[s]       even CTA only: its producer arms it with the bytes of both
//                 CTAs' loads; the odd CTA's loads complete on it remotely
//   empty[s]      one per CTA: the MMA issuer's commit releases stage s in
//                 both CTAs (one commit per barrier)
//   tmem_full[b]  one per CTA: committed by the MMA issuer to both
//   tmem_empty[b] even CTA only: the 16 epilogue warps of both CTAs arrive
//                 once they have drained accumulator buffer b
// Every wait is bounded; an abort is also stored into the peer's flag.
//
// Alg. 2 / Eq. 14 with both parts scaled by 2^s (Eq. 12: hi = fp16(Y),
// lo' = fp16(2^s (Y - hi)); hp = 2^s hi is exact in FP16 for |Y| < 2^(15-s)):
//     2^(2s) P = hp hp + lo' hp + hp lo',
// so only two FP16 planes are stored and loaded, and the three products
// accumulate into one FP32 accumulator of 256 columns; scaling by powers of
// two commutes with every rounding.  Two accumulators fill the 512 TMEM
// columns: the epilogue of tile t runs under the MMAs of tile t+1.
//
// CTA = 11 warps, persistent over the super-tile list (one CTA per SM):
//   warp 0      TMA producer (one thread)
//   warp 1      TMEM allocation (both CTAs) + MMA issuer (even CTA, one thread)
//   warps 2..9  epilogue of the CTA's 128 rows (csrc/epilogue.cuh)
//   warp 10     finisher: publishes each tile's sums, runs the control steps
// Plain FP16 (split = false): hi hi only, 32 KB stages, 6 stages.
//
// Wide units (SqArgs::wide, the single solve at large N): a pair takes the
// super tiles (I, J) and (I, J + 1) of a row together, one per accumulator,
// and loads their common A half once per K stage: a quarter fewer operand
// bytes per FLOP, at the price of an epilogue that no longer overlaps the
// next unit's MMAs.
//
// Operand reads use only the upper super tiles of the planes: a 64-wide K
// block left of the diagonal (super column k < I for the A rows of super row
// I, k < J for B) is read from the stored block (k, I) or (k, J) transposed,
// as two 64 x 64 TMA boxes per 128-row half and an MN-major shared-memory
// descriptor, with the operand's major bit set in the instruction descriptor
// for that K block.  So the planes need only be written for the upper super
// tiles (SqArgs::tri_planes).
#include <cuda.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"
#include "epilogue.cuh"

namespace sp2 {
namespace tc2 {

using namespace sp2::tc;

constexpr int BH = BM;                     // 128 rows per CTA of each operand
constexpr int HALF_BYTES = BH * BK * 2;    // 16 KB: one plane of one operand half
constexpr int STAGE_SPLIT = 4 * HALF_BYTES;  // 64 KB: hpA loA hpB loB
constexpr int STAGE_PLAIN = 2 * HALF_BYTES;  // 32 KB: hiA hiB
constexpr int STAGES_SPLIT = 3;
constexpr int STAGES_PLAIN = 6;
// Wide units (SqArgs::wide): a pair computes the super tiles (I, J) and
// (I, J + 1) together, loading the A half once per K stage for both: a stage
// holds A, B of J and B of J + 1 (96 KB split, two stages; 48 KB plain, four),
// the same 192 KB as the three 64 KB stages of one super tile.  The two
// accumulators are the two products of the unit, so the epilogue of a unit
// no longer runs under the MMAs of the next; the operand bytes per FLOP fall
// by a quarter.
constexpr int STAGE_WSPLIT = 6 * HALF_BYTES;
constexpr int STAGE_WPLAIN = 3 * HALF_BYTES;
constexpr int STAGES_WSPLIT = 2;
constexpr int STAGES_WPLAIN = 4;
constexpr int EPI_WARPS = epi::WARPS;
constexpr int FIN_WARP = 2 + EPI_WARPS;  // the finisher warp (after the epilogue warps)
constexpr int THREADS = 64 + 32 * EPI_WARPS + 32;
constexpr uint32_t TMEM_COLS = 512;  // two 256-column accumulators

// Instruction descriptor of the pair MMA: M = 256 (bits 24-28 = M >> 4),
// N = 256 (bits 17-22 = N >> 3), D = F32, A = B = F16, K-major unless the
// MN bits are added.
constexpr uint32_t IDESC2 = (1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)((2 * BM) >> 4) << 24);
// N = 128 for super tiles whose columns from J * 256 + 128 on all lie past
// the matrix (the last super column of an instance with N mod 256 in
// (0, 128]): each CTA supplies 64 B rows, the accumulator's columns 128-255
// are not written and the epilogue, which skips columns past the padded K
// extent, never reads them.
constexpr uint32_t IDESC2_N128 = (1u << 4) | ((uint32_t)(BH >> 3) << 17) | ((uint32_t)((2 * BM) >> 4) << 24);

// MMA N of super tile column J of an instance of size N
__device__ __forceinline__ int pair_n(int N, int J) { return N - J * BN <= BH ? BH : BN; }

// one 64 x 64 FP16 box of a transposed read
constexpr int T_BOX = 64 * 64 * 2;
// stage offsets (split): hpA, loA, hpB, loB
constexpr int OFF_HPA = 0, OFF_LOA = HALF_BYTES, OFF_HPB = 2 * HALF_BYTES, OFF_LOB = 3 * HALF_BYTES;
// wide units: the second B half (J + 1) after the first (split: hp, lo'; plain: hi)
constexpr int OFF_HPB1 = 4 * HALF_BYTES, OFF_LOB1 = 5 * HALF_BYTES, OFF_B1_PLAIN = 2 * HALF_BYTES;

// Loads one 128-row operand half of K block k0 into dst: K-major (one box of
// 64 x 128) when the block lies on or right of the diagonal, else the stored
// block transposed (two boxes of 64 x 64).
__device__ __forceinline__ void load_half(uint8_t* dst, const CUtensorMap* tmK, const CUtensorMap* tmT, bool trans,
                                          int row, int k0, int b, uint32_t bar_cl) {
  if (!trans) {
    tma_load_3d_pair(dst, tmK, k0, row, b, bar_cl);
  } else {
    tma_load_3d_pair(dst, tmT, row, k0, b, bar_cl);
    tma_load_3d_pair(dst + T_BOX, tmT, row + 64, k0, b, bar_cl);
  }
}

// Number of pairs with at least one K stage in epoch e (W stages each) when
// pair c takes super tiles c, c + ncl, ... of nsuper, each of nk stages (one
// instance, every tile active).
__device__ __forceinline__ unsigned pairs_in_epoch(uint32_t e, int W, int nk, int nsuper, int ncl) {
  const long long first = (long long)e * W;  // first stage of the epoch
  const int q = nsuper / ncl, r = nsuper % ncl;
  if (first < (long long)q * nk) return (unsigned)min(ncl, nsuper);
  if (first < (long long)(q + 1) * nk) return (unsigned)r;
  return 0u;
}

// Waits until *ctr >= need; false (stop waiting for the rest of the launch)
// once the wait has taken longer than a small fraction of the wait bound.
__device__ __forceinline__ bool epoch_wait(const unsigned* ctr, unsigned need, unsigned long long lim) {
  const volatile unsigned* c = ctr;
  if (*c >= need) return true;
  const unsigned long long give_up = lim / 16 < 250000ull ? lim / 16 : 250000ull;  // <= 250 us
  const uint64_t t0 = globaltimer();
  while (*c < need) {
    if (globaltimer() - t0 > give_up) return false;
  }
  return true;
}

// RO: readout mode of the epilogue (finite-temperature expansion).
// NSEG2: P = A_1 B_1^T + A_2 B_2^T over two K segments (the tm2 maps hold the
// second segment's operands) with the adjoint-mode epilogue: the split SYR2K
// Y G + G Y of the network adjoint (both factors symmetric).
// tm_p0A/p1A: planes with 64 x 128 boxes (the A half); tm_p0B/p1B: the same
// boxes for the B half; tm_p0T / tm_p1T: 64 x 64 boxes (transposed reads).
// The kernel body; the map arguments point at the kernels' __grid_constant__
// parameters (for one segment the second set repeats the first).
template <bool SPLIT, bool RO, bool NSEG2, bool WIDE>
__device__ __forceinline__ void syrk_tc2_body(const CUtensorMap& tm_p0A, const CUtensorMap& tm_p1A,
                                              const CUtensorMap& tm_p0B, const CUtensorMap& tm_p1B,
                                              const CUtensorMap& tm_p0T, const CUtensorMap& tm_p1T,
                                              const CUtensorMap& tm2_p0A, const CUtensorMap& tm2_p1A,
                                              const CUtensorMap& tm2_p0B, const CUtensorMap& tm2_p1B,
                                              const CUtensorMap& tm2_p0T, const CUtensorMap& tm2_p1T,
                                              const SqArgs& a) {
  constexpr int STAGES = WIDE ? (SPLIT ? STAGES_WSPLIT : STAGES_WPLAIN) : (SPLIT ? STAGES_SPLIT : STAGES_PLAIN);
  constexpr int STAGE_BYTES = WIDE ? (SPLIT ? STAGE_WSPLIT : STAGE_WPLAIN) : (SPLIT ? STAGE_SPLIT : STAGE_PLAIN);
  constexpr int UW = WIDE ? 2 : 1;  // super tiles per unit of work of a pair
  static_assert(!WIDE || (!RO && !NSEG2), "wide units serve the single solve");

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
  __shared__ int s_work;
  __shared__ epi::Shared s_epi;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const uint32_t peer = rank ^ 1u;

  // A pair whose super tiles all belong to finished instances (the launches
  // after a solve's last layer) leaves before any set-up; one warp looks at
  // 32 of its tiles at a time.  Both CTAs of the pair reach the same answer:
  // an instance can finish within this launch only after all of its tiles,
  // these among them, have been processed.
  if (warp == 0) {
    const int c0 = (int)(blockIdx.x >> 1), nc = (int)(gridDim.x >> 1), ns = (a.ntiles >> 1) / UW;
    bool any = false;
    for (int u0 = c0; u0 < ns && !any; u0 += 32 * nc) {
      const int u = u0 + lane * nc;
      bool act = false;
      if (u < ns) {
        int b, I, J, h;
        unpack_tile(a.tiles[2 * UW * u], b, I, J, h);
        act = load_params(a, b).active != 0;
      }
      any = __any_sync(0xffffffffu, act);
    }
    if (lane == 0) s_work = any ? 1 : 0;
  }
  __syncthreads();
  if (!s_work) return;

  if (threadIdx.x == 0) {
    s_abort = 0;
    epi::init(s_epi);
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);   // the even CTA's producer arrive (+ bytes of both CTAs)
      mbar_init(&empty[s], 1);  // one commit of the MMA issuer
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tmem_full[i], 1);
      mbar_init(&tmem_empty[i], 2 * EPI_WARPS);  // epilogue warps of both CTAs
    }
    mbar_init(drain, 1);
    mbar_init(never, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc_pair(tmem_slot, TMEM_COLS);
    tmem_relinquish_pair();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // the peer's barriers must exist before any load, commit or arrive reaches them
  cluster_sync();
  const uint32_t tmem_base = *tmem_slot;
  volatile int* abort_flag = &s_abort;
  const unsigned long long lim = wait_limit(a);
  const uint32_t peer_abort = mapa_u32(smem_u32(&s_abort), peer);
  const int cl = blockIdx.x >> 1, ncl = gridDim.x >> 1;
  const int nsuper = a.ntiles >> 1;
  const int nunits = nsuper / UW;  // a pair takes units cl, cl + ncl, ...

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      const uint32_t full_cl = mapa_u32(smem_u32(&full[0]), 0);  // the even CTA's barriers
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      uint32_t armed[STAGES];
#pragma unroll
      for (int s = 0; s < STAGES; ++s) armed[s] = 0;
      // soft synchronisation of the pairs (even CTA): gs counts this pair's K
      // stages over the launch, an epoch is W of them
      const int W = a.sync_stages;
      bool wait_sync = rank == 0 && a.wave_ctr != nullptr && W > 0;
      const bool pub_sync = wait_sync;
      uint32_t gs = 0;
      for (int u = cl; u < nunits && ok; u += ncl) {
        int b, I, J, h;
        unpack_tile(a.tiles[2 * UW * u + (int)rank], b, I, J, h);
        if (!load_params(a, b).active) continue;
        const int N = a.Ns[b];
        // each CTA supplies half of the MMA's N rows of B
        const int rowA = I * BN + (int)rank * BH, rowB = J * BN + (int)rank * (pair_n(N, J) >> 1);
        // wide units: the second super tile (I, J1), or none (a row's odd last tile)
        int J1 = 0, rowB1 = 0;
        bool two = false;
        if (WIDE) {
          int b1, I1, h1;
          unpack_tile(a.tiles[2 * UW * u + 2 + (int)rank], b1, I1, J1, h1);
          two = I1 * BN < N;
          rowB1 = J1 * BN + (int)rank * (pair_n(N, J1) >> 1);
        }
        const int nk = (N + BK - 1) / BK;
        const int nkt = NSEG2 ? 2 * nk : nk;  // K stages of the tile over both segments
        const bool rev = a.snake && (((u - cl) / ncl) & 1);
        for (int kk = 0; kk < nkt; ++kk, ++gs) {
          const int kbt = rev ? nkt - 1 - kk : kk;
          const bool seg2 = NSEG2 && kbt >= nk;
          const int kb = seg2 ? kbt - nk : kbt;  // K block within its segment
          if (pub_sync && gs > 0 && gs % (uint32_t)W == 0) {
            const uint32_t e = gs / (uint32_t)W - 1u;  // the epoch this pair just finished
            atomicAdd(&a.wave_ctr[e], 1u);
            if (wait_sync && e >= 1u)
              wait_sync = epoch_wait(a.wave_ctr + (e - 1u), pairs_in_epoch(e - 1u, W, nkt, nunits, ncl), lim);
          }
          if (!mbar_wait_cl(&empty[stage], phase ^ 1u, abort_flag, lim)) {
            ok = false;
            break;
          }
          uint8_t* st = smem + stage * STAGE_BYTES;
          if (rank == 0) {
            // a wide unit without its second tile loads no second B half
            const int bytes = (WIDE && !two) ? STAGE_BYTES - (SPLIT ? 2 : 1) * HALF_BYTES : STAGE_BYTES;
            mbar_expect_tx(&full[stage], 2 * bytes);
            ++armed[stage];
          }
          const uint32_t bar = full_cl + 8u * (uint32_t)stage;
          const int k0 = kb * BK;
          const int ks = k0 / BN;  // super column of this K block
          // the second segment's A and B come from the other matrix of the
          // product (their transposed reads too)
          const CUtensorMap* mA0 = seg2 ? &tm2_p0A : &tm_p0A;
          const CUtensorMap* mA1 = seg2 ? &tm2_p1A : &tm_p1A;
          const CUtensorMap* mB0 = seg2 ? &tm2_p0B : &tm_p0B;
          const CUtensorMap* mB1 = seg2 ? &tm2_p1B : &tm_p1B;
          const CUtensorMap* mAT0 = seg2 ? &tm2_p0T : &tm_p0T;
          const CUtensorMap* mAT1 = seg2 ? &tm2_p1T : &tm_p1T;
          const CUtensorMap* mBT0 = NSEG2 ? (seg2 ? &tm_p0T : &tm2_p0T) : &tm_p0T;
          const CUtensorMap* mBT1 = NSEG2 ? (seg2 ? &tm_p1T : &tm2_p1T) : &tm_p1T;
          if (SPLIT) {
            load_half(st + OFF_HPA, mA0, mAT0, ks < I, rowA, k0, b, bar);
            load_half(st + OFF_LOA, mA1, mAT1, ks < I, rowA, k0, b, bar);
            load_half(st + OFF_HPB, mB0, mBT0, ks < J, rowB, k0, b, bar);
            load_half(st + OFF_LOB, mB1, mBT1, ks < J, rowB, k0, b, bar);
            if (WIDE && two) {
              load_half(st + OFF_HPB1, mB0, mBT0, ks < J1, rowB1, k0, b, bar);
              load_half(st + OFF_LOB1, mB1, mBT1, ks < J1, rowB1, k0, b, bar);
            }
          } else {
            load_half(st, mA0, mAT0, ks < I, rowA, k0, b, bar);
            load_half(st + HALF_BYTES, mB0, mBT0, ks < J, rowB, k0, b, bar);
            if (WIDE && two) load_half(st + OFF_B1_PLAIN, mB0, mBT0, ks < J1, rowB1, k0, b, bar);
          }
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      // the last (possibly partial) epoch of this pair
      if (pub_sync && gs > 0) atomicAdd(&a.wave_ctr[(gs - 1u) / (uint32_t)W], 1u);
      if (!ok || *abort_flag) {
        atomicExch(a.err, (int)SP2_ERR_DEVICE_TIMEOUT);
        st_cluster_u32(peer_abort, 1u);
        if (rank == 0) {
          // the armed phases complete once both CTAs' bytes have landed
          for (int s = 0; s < STAGES; ++s) {
            if (armed[s] == 0) continue;
            const uint64_t t0 = globaltimer();
            while (!mbar_try_wait_cl(&full[s], (armed[s] - 1u) & 1u) && globaltimer() - t0 < lim) {
            }
          }
        } else {
          // the odd CTA's loads complete on the even CTA's barriers, which it
          // cannot poll: give its last loads time to land before it leaves
          const uint64_t t0 = globaltimer();
          while (globaltimer() - t0 < 2000000ull) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0 && rank == 0) {
      const uint32_t empty_own = smem_u32(&empty[0]);
      const uint32_t empty_peer = mapa_u32(empty_own, 1);
      const uint32_t tfull_own = smem_u32(&tmem_full[0]);
      const uint32_t tfull_peer = mapa_u32(tfull_own, 1);
      int stage = 0;
      uint32_t phase = 0, it = 0;
      bool ok = true, issued = false;
      // injected fault (SqArgs::stall): a wait that runs out after lim
      if (a.stall && !mbar_wait(never, 0, abort_flag, lim)) ok = false;
      for (int u = cl; u < nunits && ok; u += ncl) {
        int b, I, J, h;
        unpack_tile(a.tiles[2 * UW * u], b, I, J, h);
        if (!load_params(a, b).active) continue;
        const int N = a.Ns[b];
        const int nk = (N + BK - 1) / BK;
        const int nkt = NSEG2 ? 2 * nk : nk;
        const bool rev = a.snake && (((u - cl) / ncl) & 1);
        // wide units: the second super tile (I, J1) into the other accumulator
        int J1 = 0;
        bool two = false;
        if (WIDE) {
          int b1, I1, h1;
          unpack_tile(a.tiles[2 * UW * u + 2], b1, I1, J1, h1);
          two = I1 * BN < N;
        }
        const uint32_t buf = it & 1u;  // wide units: it is even, both buffers are used
        const uint32_t idesc_n = pair_n(N, J) == BH ? IDESC2_N128 : IDESC2;
        const uint32_t idesc_n1 = pair_n(N, J1) == BH ? IDESC2_N128 : IDESC2;
        (void)h;
        // the k-th use of a buffer waits for the epilogues' (k-1)-th release
        bool got = mbar_wait_cl(&tmem_empty[buf], ((it >> 1) & 1u) ^ 1u, abort_flag, lim);
        if (WIDE && got) got = mbar_wait_cl(&tmem_empty[1], ((it >> 1) & 1u) ^ 1u, abort_flag, lim);
        if (!got) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem_base + buf * BN;
        const uint32_t d1 = tmem_base + BN;  // wide units: the second accumulator
        for (int kk = 0; kk < nkt; ++kk) {
          const int kbt = rev ? nkt - 1 - kk : kk;
          const int kb = (NSEG2 && kbt >= nk) ? kbt - nk : kbt;  // K block within its segment
          if (!mbar_wait_cl(&full[stage], phase, abort_flag, lim)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = smem_u32(smem + stage * STAGE_BYTES);
          // operands left of the diagonal arrived transposed (MN-major)
          const int sc = kb * BK / BN;
          const bool ta = sc < I, tb = sc < J;
          const uint32_t idesc = idesc_n | (ta ? IDESC_A_MN : 0u) | (tb ? IDESC_B_MN : 0u);
          const bool tb1 = sc < J1;
          const uint32_t idesc1 = idesc_n1 | (ta ? IDESC_A_MN : 0u) | (tb1 ? IDESC_B_MN : 0u);
#pragma unroll
          for (int ks = 0; ks < BK / UMMA_K; ++ks) {
            // K step ks: 32 B along a K-major row, or two 8-row K groups
            const uint32_t oa = ta ? ks * 2048u : ks * UMMA_K * 2u;
            const uint32_t ob = tb ? ks * 2048u : ks * UMMA_K * 2u;
            const uint32_t ob1 = tb1 ? ks * 2048u : ks * UMMA_K * 2u;
            const uint32_t acc = (kk > 0 || ks > 0) ? 1u : 0u;
            if (SPLIT) {
              const uint64_t dhpA = ta ? make_desc_mn128(st + OFF_HPA + oa) : make_desc_sw128(st + OFF_HPA + oa);
              const uint64_t dloA = ta ? make_desc_mn128(st + OFF_LOA + oa) : make_desc_sw128(st + OFF_LOA + oa);
              const uint64_t dhpB = tb ? make_desc_mn128(st + OFF_HPB + ob) : make_desc_sw128(st + OFF_HPB + ob);
              const uint64_t dloB = tb ? make_desc_mn128(st + OFF_LOB + ob) : make_desc_sw128(st + OFF_LOB + ob);
              mma_f16_pair(d, dhpA, dhpB, idesc, acc);  // hp hp
              mma_f16_pair(d, dloA, dhpB, idesc, 1u);   // lo' hp
              mma_f16_pair(d, dhpA, dloB, idesc, 1u);   // hp lo'
              if (WIDE && two) {
                const uint64_t dhpB1 =
                    tb1 ? make_desc_mn128(st + OFF_HPB1 + ob1) : make_desc_sw128(st + OFF_HPB1 + ob1);
                const uint64_t dloB1 =
                    tb1 ? make_desc_mn128(st + OFF_LOB1 + ob1) : make_desc_sw128(st + OFF_LOB1 + ob1);
                mma_f16_pair(d1, dhpA, dhpB1, idesc1, acc);
                mma_f16_pair(d1, dloA, dhpB1, idesc1, 1u);
                mma_f16_pair(d1, dhpA, dloB1, idesc1, 1u);
              }
            } else {
              const uint64_t dA = ta ? make_desc_mn128(st + oa) : make_desc_sw128(st + oa);
              const uint64_t dB = tb ? make_desc_mn128(st + HALF_BYTES + ob) : make_desc_sw128(st + HALF_BYTES + ob);
              mma_f16_pair(d, dA, dB, idesc, acc);
              if (WIDE && two) {
                const uint64_t dB1 = tb1 ? make_desc_mn128(st + OFF_B1_PLAIN + ob1)
                                         : make_desc_sw128(st + OFF_B1_PLAIN + ob1);
                mma_f16_pair(d1, dA, dB1, idesc1, acc);
              }
            }
          }
          // release the stage in both CTAs
          mma_commit_pair(empty_own + 8u * (uint32_t)stage);
          mma_commit_pair(empty_peer + 8u * (uint32_t)stage);
          issued = true;
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        mma_commit_pair(tfull_own + 8u * buf);
        mma_commit_pair(tfull_peer + 8u * buf);
        if (WIDE) {
          // also when the unit has no second tile: its epilogue waits for it
          mma_commit_pair(tfull_own + 8u);
          mma_commit_pair(tfull_peer + 8u);
        }
        it += UW;
      }
      if (!ok || *abort_flag) {
        atomicExch(a.err, (int)SP2_ERR_DEVICE_TIMEOUT);
        st_cluster_u32(peer_abort, 1u);
      }
      if (issued) {
        mma_commit_pair(smem_u32(drain));
        const uint64_t t0 = globaltimer();
        while (!mbar_try_wait(drain, 0) && globaltimer() - t0 < lim) {
        }
      }
    }
  } else if (warp == FIN_WARP) {
    // ------------------------------------------------------------ finisher
    // (tiles t = 2 (UW u + k) + rank of units u = cl, cl + ncl, ...)
    epi::finisher_pair(a, cl, ncl, nunits, UW, (int)rank, s_epi, abort_flag, lane);
    if (*abort_flag && lane == 0) st_cluster_u32(peer_abort, 1u);
  } else {
    // ------------------------------------------------------------ epilogue
    const int ew = warp - 2;  // 0..7
    const int q = warp & 3;   // TMEM lane quarter
    const uint32_t empty_cl = mapa_u32(smem_u32(&tmem_empty[0]), 0);
    uint32_t it = 0;
    bool ok = true;
    for (int u = cl; u < nunits && ok; u += ncl) {
      // a unit's super tiles use the accumulator buffers in turn (a wide
      // unit's second tile, when it has none, has no rows to store)
      for (int k = 0; k < UW; ++k) {
        const int t = 2 * (UW * u + k) + (int)rank;
        const int rc = epi::tile<SPLIT, NSEG2, RO, true>(a, t, it, tmem_base, tmem_full, tmem_empty, abort_flag,
                                                          s_epi, ew, q, lane, trbuf + ew * epi::TR_FLOATS, empty_cl);
        if (rc < 0) {
          if (lane == 0) st_cluster_u32(peer_abort, 1u);
          ok = false;
          break;
        }
        it += (uint32_t)rc;
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // neither CTA leaves (or frees its tensor memory) while the pair's MMAs,
  // loads or arrivals may still reach it
  cluster_sync();
  if (warp == 1) {
    __syncwarp();
    tmem_dealloc_pair(tmem_base, TMEM_COLS);
  }
}

template <bool SPLIT, bool RO>
__global__ void __launch_bounds__(THREADS, 1)
    syrk_tc2_kernel(const __grid_constant__ CUtensorMap tm_p0A, const __grid_constant__ CUtensorMap tm_p1A,
                    const __grid_constant__ CUtensorMap tm_p0B, const __grid_constant__ CUtensorMap tm_p1B,
                    const __grid_constant__ CUtensorMap tm_p0T, const __grid_constant__ CUtensorMap tm_p1T,
                    const SqArgs a) {
  syrk_tc2_body<SPLIT, RO, false, false>(tm_p0A, tm_p1A, tm_p0B, tm_p1B, tm_p0T, tm_p1T, tm_p0A, tm_p1A, tm_p0B,
                                         tm_p1B, tm_p0T, tm_p1T, a);
}

// Wide units (the single solve): super tiles (I, J) and (I, J + 1) per pass.
template <bool SPLIT>
__global__ void __launch_bounds__(THREADS, 1)
    syrk_tc2_wide_kernel(const __grid_constant__ CUtensorMap tm_p0A, const __grid_constant__ CUtensorMap tm_p1A,
                         const __grid_constant__ CUtensorMap tm_p0B, const __grid_constant__ CUtensorMap tm_p1B,
                         const __grid_constant__ CUtensorMap tm_p0T, const __grid_constant__ CUtensorMap tm_p1T,
                         const SqArgs a) {
  syrk_tc2_body<SPLIT, false, false, true>(tm_p0A, tm_p1A, tm_p0B, tm_p1B, tm_p0T, tm_p1T, tm_p0A, tm_p1A, tm_p0B,
                                           tm_p1B, tm_p0T, tm_p1T, a);
}

// Two K segments (the network adjoint's Y G + G Y): six maps per segment.
template <bool SPLIT>
__global__ void __launch_bounds__(THREADS, 1)
    syrk_tc2_seg2_kernel(const __grid_constant__ CUtensorMap tm_p0A, const __grid_constant__ CUtensorMap tm_p1A,
                         const __grid_constant__ CUtensorMap tm_p0B, const __grid_constant__ CUtensorMap tm_p1B,
                         const __grid_constant__ CUtensorMap tm_p0T, const __grid_constant__ CUtensorMap tm_p1T,
                         const __grid_constant__ CUtensorMap tm2_p0A, const __grid_constant__ CUtensorMap tm2_p1A,
                         const __grid_constant__ CUtensorMap tm2_p0B, const __grid_constant__ CUtensorMap tm2_p1B,
                         const __grid_constant__ CUtensorMap tm2_p0T, const __grid_constant__ CUtensorMap tm2_p1T,
                         const SqArgs a) {
  syrk_tc2_body<SPLIT, false, true, false>(tm_p0A, tm_p1A, tm_p0B, tm_p1B, tm_p0T, tm_p1T, tm2_p0A, tm2_p1A, tm2_p0B,
                                           tm2_p1B, tm2_p0T, tm2_p1T, a);
}

}  // namespace tc2

// The dynamic shared-memory opt-in, once per kernel and device (not a stream
// operation, and kept out of captured launch sequences).
namespace {
template <typename K>
cudaError_t set_smem_once(K kernel, int bytes, int which) {
  static int done_dev[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
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
  static_assert(tc2::STAGES_WSPLIT * tc2::STAGE_WSPLIT == tc2::STAGES_SPLIT * tc2::STAGE_SPLIT &&
                    tc2::STAGES_WPLAIN * tc2::STAGE_WPLAIN == tc2::STAGES_PLAIN * tc2::STAGE_PLAIN,
                "wide units use the same shared memory as single super tiles");
  return (size_t)stages * sb + 1024 /* alignment slack */ + 256 /* barriers */ + epi::TR_BYTES;
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
  auto go = [&](auto kernel, int which) -> cudaError_t {
    cudaError_t e = set_smem_once(kernel, (int)smem, which);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernelEx(&cfg, kernel, tm[0], tm[1], tm[2], tm[3], tm[4], tm[5], a);
  };
  auto go2 = [&](auto kernel, int which) -> cudaError_t {
    cudaError_t e = set_smem_once(kernel, (int)smem, which);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernelEx(&cfg, kernel, tm[0], tm[1], tm[2], tm[3], tm[4], tm[5], tm[6], tm[7], tm[8], tm[9],
                              tm[10], tm[11], a);
  };
  cudaError_t e;
  if (a.nseg == 2)
    e = split ? go2(tc2::syrk_tc2_seg2_kernel<true>, 5) : go2(tc2::syrk_tc2_seg2_kernel<false>, 4);
  else if (a.wide)
    e = split ? go(tc2::syrk_tc2_wide_kernel<true>, 7) : go(tc2::syrk_tc2_wide_kernel<false>, 6);
  else if (a.R)
    e = split ? go(tc2::syrk_tc2_kernel<true, true>, 3) : go(tc2::syrk_tc2_kernel<false, true>, 2);
  else
    e = split ? go(tc2::syrk_tc2_kernel<true, false>, 1) : go(tc2::syrk_tc2_kernel<false, false>, 0);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace sp2
