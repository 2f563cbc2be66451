// Per-tile completion of the squaring kernels: each tile publishes its FP64
// (tr Y', ||Y'||_F^2) partial; the warp that completes the last tile of an
// instance sums that instance's partials in tile order (deterministic) and
// runs the instance's SP2 control step (or stores the traces).
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace sp2 {

// Warp-collective: all 32 lanes of one warp call it; (tr, sq) valid in lane 0.
// With a control block: a final (OUT_D) launch, or any launch with fused_ctl
// set, runs the control step here; otherwise tr Y' is left for the row-norm
// launch, which owns ||Y'||_F^2 and runs the control step.
__device__ inline void finish_tile_warp(const SqArgs& a, int t, int b, double tr, double sq, int out_mode) {
  const int lane = threadIdx.x & 31;
  unsigned last = 0;
  if (lane == 0) {
    a.tile_part[t] = make_double2(tr, sq);
    __threadfence();
    const unsigned done = atomicAdd(&a.inst_done[b], 1u);
    last = (done == (unsigned)a.tile_cnt[b] - 1u) ? 1u : 0u;
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (!last) return;
  __threadfence();
  const int off = a.tile_off[b], cnt = a.tile_cnt[b];
  double T = 0.0, Q = 0.0;
#pragma unroll 4
  for (int k = lane; k < cnt; k += 32) {
    const double2 p = __ldcg(&a.tile_part[off + k]);
    T += p.x;
    Q += p.y;
  }
  T = warp_sum_d(T);
  Q = warp_sum_d(Q);
  double d0 = 0.0, d1 = 0.0, d2 = 0.0;
  // per-tile dots exist in adjoint mode and, for Tr[D A], in the launch that writes D
  const bool dots = a.dots_out && (a.aux || (a.Hobs && out_mode == OUT_D));
  if (dots) {
    for (int k = lane; k < cnt; k += 32) {
      const double* td = a.tile_dots + 3 * (long long)(off + k);
      d0 += __ldcg(td);
      d1 += __ldcg(td + 1);
      d2 += __ldcg(td + 2);
    }
    d0 = warp_sum_d(d0);
    d1 = warp_sum_d(d1);
    d2 = warp_sum_d(d2);
  }
  if (lane == 0) {
    if (dots) {
      a.dots_out[3 * b + 0] = d0;
      a.dots_out[3 * b + 1] = d1;
      a.dots_out[3 * b + 2] = d2;
    }
    a.inst_done[b] = 0u;
    if (a.ctl) {
      if (out_mode == OUT_D || a.fused_ctl)
        control_step(a.ctl + b, T, Q);
      else
        a.ctl[b].trY_new = T;
    } else if (a.traces_out) {
      a.traces_out[2 * b] = T;
      a.traces_out[2 * b + 1] = Q;
    }
  }
}

}  // namespace sp2
