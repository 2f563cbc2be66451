// Memory-bound kernels of the SP2 path (sm_103a):
//   K1 gershgorin_kernel   spectral bound estimates (Alg. 1 inputs), FP64
//   K2 input_layer_kernel  S_0 = W_0 H + B_0 (Alg. 1), stored as alpha_0 I + Y_0,
//                          FP16 split of Y_0 (Eq. 12), FP64 trace partials,
//                          then the first control step (sigma_1, IdErr_1)
//      split_kernel        stand-alone split (Eq. 12)
//      observable_kernel   Tr[D A] (Alg. 1, last line)
//      network prologue    the same input layer for a batch, no control
#include <cuda_fp16.h>
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace sp2 {

// ---------------------------------------------------------------- K1
// One warp per row: R_i = sum_j |H_ij| - |H_ii|.  Groups of sixteen are
// summed in FP32 as a four-level tree (relative error <= 4 x 2^-24) and
// accumulated in FP64 (GB300's FP64 rate, not memory, would otherwise bound
// the pass).  Per-block min/max, then
// the last block folds all blocks and writes the bounds into each
// instance's control block (or bounds_out).
__global__ void __launch_bounds__(256) gershgorin_kernel(const float* __restrict__ H, int N, long long ld,
                                                         long long slot, int B, double2* __restrict__ partials,
                                                         unsigned* __restrict__ ticket, Ctl* ctl,
                                                         double* bounds_out, long long nan_row) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long rows_total = (long long)N * B;
  double lo = INFINITY, hi = -INFINITY;
  const bool vec = ((ld & 3) == 0) && ((((uintptr_t)H) & 15) == 0);
  bool bad = false;
  for (long long gr = (long long)blockIdx.x * 8 + warp; gr < rows_total; gr += (long long)gridDim.x * 8) {
    const int b = (int)(gr / N), i = (int)(gr % N);
    const float* row = H + (long long)b * slot + (long long)i * ld;
    double acc = 0.0;
    if (vec) {
      // four independent loads and FP64 accumulators per step (the FP64
      // adds would otherwise serialise the row)
      const float4* r4 = reinterpret_cast<const float4*>(row);
      const int n4 = N >> 2;
      double a4[4] = {0.0, 0.0, 0.0, 0.0};
      int j = lane;
      for (; j + 96 < n4; j += 128) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = __ldcs(r4 + j + 32 * u);
        float g4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) g4[u] = (fabsf(v[u].x) + fabsf(v[u].y)) + (fabsf(v[u].z) + fabsf(v[u].w));
        // the four groups in FP32 (a four-level tree of 16 terms), then FP64
        a4[1] += (double)((g4[0] + g4[1]) + (g4[2] + g4[3]));
      }
      for (; j < n4; j += 32) {
        const float4 v = __ldcs(r4 + j);
        a4[0] += (double)((fabsf(v.x) + fabsf(v.y)) + (fabsf(v.z) + fabsf(v.w)));
      }
      acc = (a4[0] + a4[1]) + (a4[2] + a4[3]);
      for (int jj = (n4 << 2) + lane; jj < N; jj += 32) acc += (double)fabsf(row[jj]);
    } else {
      for (int j = lane; j < N; j += 32) acc += (double)fabsf(row[j]);
    }
    acc = warp_sum_d(acc);
    const double d = (double)row[i];
    const double R = acc - fabs(d);
    if (!isfinite(R) || !isfinite(d)) bad = true;  // fmin/fmax would drop a NaN
    if (gr == nan_row) bad = true;                    // injected fault: this row reads as holding a NaN
    lo = fmin(lo, d - R);
    hi = fmax(hi, d + R);
  }
  __shared__ double s_lo[8], s_hi[8];
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  if (lane == 0) {
    s_lo[warp] = lo;
    s_hi[warp] = hi;
    if (bad) atomicOr(&s_bad, 1);
  }
  __syncthreads();
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
    for (int w = 0; w < 8; ++w) {
      lo = fmin(lo, s_lo[w]);
      hi = fmax(hi, s_hi[w]);
    }
    if (s_bad) lo = hi = NAN;
    partials[blockIdx.x] = make_double2(lo, hi);
    __threadfence();
    s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;
  __threadfence();
  double L = INFINITY, U = -INFINITY;
  bool nonfinite = false;
  for (unsigned k = 0; k < gridDim.x; ++k) {
    const double2 p = __ldcg(&partials[k]);
    if (isnan(p.x) || isnan(p.y)) nonfinite = true;
    L = fmin(L, p.x);
    U = fmax(U, p.y);
  }
  if (isnan(L) || isnan(U)) nonfinite = true;
  *ticket = 0u;
  if (bounds_out) {
    bounds_out[0] = nonfinite ? NAN : L;
    bounds_out[1] = nonfinite ? NAN : U;
  }
  if (ctl) {
    // single-instance path (B == 1)
    Ctl* c = ctl;
    c->e_min = L;
    c->e_max = U;
    if (nonfinite || !isfinite(L) || !isfinite(U)) {
      c->status = SP2_ERR_NONFINITE;
      c->phase = PHASE_ERROR;
      c->next.active = 0;
    } else if (!(U - L > 0.0)) {
      if (c->n_occ == 0 || c->n_occ == c->N) {
        // H = cI: any enclosing interval is a valid bound estimate
        c->e_min = L - 1.0;
        c->e_max = U + 1.0;
      } else {
        c->status = SP2_ERR_DEGENERATE_SPECTRUM;
        c->phase = PHASE_ERROR;
        c->next.active = 0;
      }
    }
  }
}

// Per-instance Gershgorin for the batched path: grid (blocks, instances),
// one warp per row as above, per-block partials, and the last block of each
// instance folds them into ctl[b].
__global__ void __launch_bounds__(256) gershgorin_batched_kernel(const float* const* __restrict__ Hs,
                                                                 const int* __restrict__ Ns, Ctl* __restrict__ ctl,
                                                                 double2* __restrict__ partials,
                                                                 unsigned* __restrict__ tickets) {
  const int b = blockIdx.y;
  const int N = Ns[b];
  const float* H = Hs[b];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool vec = ((N & 3) == 0) && ((((uintptr_t)H) & 15) == 0);
  double lo = INFINITY, hi = -INFINITY;
  bool bad = false;
  for (int i = blockIdx.x * 8 + warp; i < N; i += gridDim.x * 8) {
    const float* row = H + (long long)i * N;
    double acc = 0.0;
    if (vec) {
      const float4* r4 = reinterpret_cast<const float4*>(row);
      const int n4 = N >> 2;
      for (int j0 = 0; j0 < n4; j0 += 4 * 32) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = j0 + u * 32 + lane;
          v[u] = (j < n4) ? __ldcs(r4 + j) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float g4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) g4[u] = (fabsf(v[u].x) + fabsf(v[u].y)) + (fabsf(v[u].z) + fabsf(v[u].w));
        // sixteen terms as an FP32 tree, one FP64 add (as the single-matrix kernel)
        acc += (double)((g4[0] + g4[1]) + (g4[2] + g4[3]));
      }
    } else {
      for (int j = lane; j < N; j += 32) acc += (double)fabsf(row[j]);
    }
    acc = warp_sum_d(acc);
    const double d = (double)row[i];
    const double R = acc - fabs(d);
    if (!isfinite(R) || !isfinite(d)) bad = true;
    lo = fmin(lo, d - R);
    hi = fmax(hi, d + R);
  }
  __shared__ double s_lo[8], s_hi[8];
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  if (lane == 0) {
    s_lo[warp] = lo;
    s_hi[warp] = hi;
    if (bad) atomicOr(&s_bad, 1);
  }
  __syncthreads();
  __shared__ bool s_last;
  double2* part = partials + (long long)b * gridDim.x;
  if (threadIdx.x == 0) {
    for (int w = 0; w < 8; ++w) {
      lo = fmin(lo, s_lo[w]);
      hi = fmax(hi, s_hi[w]);
    }
    if (s_bad) lo = hi = NAN;
    part[blockIdx.x] = make_double2(lo, hi);
    __threadfence();
    s_last = (atomicAdd(&tickets[b], 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;
  __threadfence();
  double L = INFINITY, U = -INFINITY;
  bool nan_seen = false;
  for (unsigned k = 0; k < gridDim.x; ++k) {
    const double2 p = __ldcg(&part[k]);
    if (isnan(p.x) || isnan(p.y)) nan_seen = true;
    L = fmin(L, p.x);
    U = fmax(U, p.y);
  }
  tickets[b] = 0u;
  Ctl* c = ctl + b;
  c->e_min = L;
  c->e_max = U;
  if (nan_seen || !isfinite(L) || !isfinite(U)) {
    c->status = SP2_ERR_NONFINITE;
    c->phase = PHASE_ERROR;
    c->next.active = 0;
  } else if (!(U - L > 0.0)) {
    if (c->n_occ == 0 || c->n_occ == c->N) {
      c->e_min = L - 1.0;
      c->e_max = U + 1.0;
    } else {
      c->status = SP2_ERR_DEGENERATE_SPECTRUM;
      c->phase = PHASE_ERROR;
      c->next.active = 0;
    }
  }
}

// ---------------------------------------------------------------- K2
// Input layer for one instance (b = blockIdx.y): y = (shift ? -h : (e_max d_ij - h)) / (e_max - e_min)
// written as FP32 into Y (ld_y, slot_y) and as the FP16 planes of Eq. 12
// (hi, lo' and/or hp = 2^s hi, whichever pointers are set; ld_h, slot_h;
// padding up to rows_pad x cols_pad zero-filled).  FP64 partial of tr Y and,
// when ctl_step, the shift of S_0 and tr Y_0 for the first control step.
__global__ void __launch_bounds__(256) input_layer_kernel(const float* const* __restrict__ Hs,
                                                          const int* __restrict__ Ns, long long ld_in_fixed,
                                                          float* __restrict__ Y, long long ld_y, long long slot_y,
                                                          __half* __restrict__ hi, __half* __restrict__ lo,
                                                          __half* __restrict__ hp, long long ld_h, long long slot_h,
                                                          int rows_pad, int cols_pad,
                                                          float lo_scale,
                                                          Ctl* __restrict__ ctl, const double* __restrict__ bounds,
                                                          double2* __restrict__ partials, unsigned* __restrict__ tickets,
                                                          int shift, int ctl_step) {
  const int b = blockIdx.y;
  const int N = Ns[b];
  const float* H = Hs[b];
  const long long ld_in = ld_in_fixed > 0 ? ld_in_fixed : N;
  double e_min, e_max;
  bool active = true;
  if (ctl) {
    const Ctl* c = ctl + b;
    active = (c->phase != PHASE_ERROR);
    e_min = c->e_min;
    e_max = c->e_max;
  } else {
    e_min = bounds[2 * b];
    e_max = bounds[2 * b + 1];
  }
  const double inv = 1.0 / (e_max - e_min);
  const double diag_add = shift ? 0.0 : e_max * inv;
  // off-diagonal y = -h inv in FP32: inv as a sum of two floats and one FMA
  // (-h inv_hi + (-h inv_lo) rounded once), the correctly rounded FP64 value
  // except within 2^-47 of a rounding boundary; the diagonal stays in FP64
  const float inv_hi = (float)inv, inv_lo = (float)(inv - (double)inv_hi);
  double tr = 0.0, sq = 0.0;
  if (active) {
    // FP16 planes: hi (plain), or hp = 2^s hi and lo' (split); hi may be absent
    const bool halves = (hi != nullptr) || (hp != nullptr);
    const int rows = halves ? rows_pad : N;
    const int cols = halves ? cols_pad : N;
    const bool vec = ((ld_in & 3) == 0) && ((ld_y & 3) == 0) && ((slot_y & 3) == 0) && ((((uintptr_t)H) & 15) == 0) &&
                     ((((uintptr_t)Y) & 15) == 0) && (!halves || ((ld_h & 3) == 0 && (slot_h & 3) == 0));
    if (vec) {
      // four consecutive columns per thread: float4 loads and stores, 8-byte plane stores
      for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const float* hrow = H + (long long)r * ld_in;
        float* yrow = Y + (long long)b * slot_y + (long long)r * ld_y;
        __half* hirow = hi ? hi + (long long)b * slot_h + (long long)r * ld_h : nullptr;
        __half* lorow = (halves && lo) ? lo + (long long)b * slot_h + (long long)r * ld_h : nullptr;
        __half* hprow = hp ? hp + (long long)b * slot_h + (long long)r * ld_h : nullptr;
        float sqf = 0.f;
        for (int c4 = threadIdx.x * 4; c4 < cols; c4 += blockDim.x * 4) {
          float y[4] = {0.f, 0.f, 0.f, 0.f};
          if (r < N) {
            float hv[4];
            if (c4 + 3 < N) {
              const float4 o = __ldcs(reinterpret_cast<const float4*>(hrow + c4));
              hv[0] = o.x;
              hv[1] = o.y;
              hv[2] = o.z;
              hv[3] = o.w;
            } else {
#pragma unroll
              for (int u = 0; u < 4; ++u) hv[u] = (c4 + u < N) ? hrow[c4 + u] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) y[u] = (c4 + u < N) ? fmaf(-hv[u], inv_hi, -hv[u] * inv_lo) : 0.f;
            // the diagonal element (at most one per group) in FP64, once
            const int du = r - c4;
            if ((unsigned)du < 4u) {
              float hd = 0.f;
#pragma unroll
              for (int u = 0; u < 4; ++u)
                if (u == du) hd = hv[u];
              const float yd = (float)(-(double)hd * inv + diag_add);
              tr += (double)yd;
#pragma unroll
              for (int u = 0; u < 4; ++u)
                if (u == du) y[u] = yd;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) sqf = fmaf(y[u], y[u], sqf);
            if (c4 + 3 < N) {
              *reinterpret_cast<float4*>(yrow + c4) = make_float4(y[0], y[1], y[2], y[3]);
            } else {
#pragma unroll
              for (int u = 0; u < 4; ++u)
                if (c4 + u < N) yrow[c4 + u] = y[u];
            }
          }
          if (halves) {
            __half h16[4], l16[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) split_fp16(y[u], lo_scale, h16[u], l16[u]);
            auto pk = [](__half x0, __half x1) {
              return (uint32_t)__half_as_ushort(x0) | ((uint32_t)__half_as_ushort(x1) << 16);
            };
            if (hirow) *reinterpret_cast<uint2*>(hirow + c4) = make_uint2(pk(h16[0], h16[1]), pk(h16[2], h16[3]));
            if (lorow) *reinterpret_cast<uint2*>(lorow + c4) = make_uint2(pk(l16[0], l16[1]), pk(l16[2], l16[3]));
            if (hprow) {
              __half p16[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) p16[u] = __float2half_rn(__half2float(h16[u]) * lo_scale);
              *reinterpret_cast<uint2*>(hprow + c4) = make_uint2(pk(p16[0], p16[1]), pk(p16[2], p16[3]));
            }
          }
        }
        sq += (double)sqf;
      }
    } else
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
      const float* hrow = H + (long long)r * ld_in;
      float* yrow = Y + (long long)b * slot_y + (long long)r * ld_y;
      __half* hirow = hi ? hi + (long long)b * slot_h + (long long)r * ld_h : nullptr;
      __half* lorow = (halves && lo) ? lo + (long long)b * slot_h + (long long)r * ld_h : nullptr;
      __half* hprow = hp ? hp + (long long)b * slot_h + (long long)r * ld_h : nullptr;
      float sqf = 0.f;
      for (int col = threadIdx.x; col < cols; col += blockDim.x) {
        float y = 0.f;
        if (r < N && col < N) {
          const float hv = hrow[col];
          if (r == col)
            y = (float)(-(double)hv * inv + diag_add);
          else
            y = fmaf(-hv, inv_hi, -hv * inv_lo);
          yrow[col] = y;
          if (r == col) tr += (double)y;
          sqf = fmaf(y, y, sqf);
        }
        if (halves) {
          __half h16, l16;
          split_fp16(y, lo_scale, h16, l16);
          if (hirow) hirow[col] = h16;
          if (lorow) lorow[col] = l16;
          if (hprow) hprow[col] = __float2half_rn(__half2float(h16) * lo_scale);
        }
      }
      sq += (double)sqf;
    }
  }
  tr = warp_sum_d(tr);
  sq = warp_sum_d(sq);
  __shared__ double s_tr[8], s_sq[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    s_tr[warp] = tr;
    s_sq[warp] = sq;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    tr = 0.0;
    sq = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      tr += s_tr[w];
      sq += s_sq[w];
    }
  }
  if (!ctl_step || ctl == nullptr) return;
  // last-block reduction per instance
  __shared__ bool s_last;
  double2* part = partials + (long long)b * gridDim.x;
  if (threadIdx.x == 0) {
    part[blockIdx.x] = make_double2(tr, sq);
    __threadfence();
    s_last = (atomicAdd(&tickets[b], 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;
  __threadfence();
  double T = 0.0, Q = 0.0;
  for (unsigned k = 0; k < gridDim.x; ++k) {
    const double2 p = __ldcg(&part[k]);
    T += p.x;
    Q += p.y;
  }
  tickets[b] = 0u;
  Ctl* c = ctl + b;
  if (!active) return;
  // S_0 = alpha_0 I + Y_0; the row-norm launch that follows runs the first
  // control step (sigma_1, IdErr_1) with the exact ||Y_0||_F^2.
  c->alpha_next = shift ? e_max * inv : 0.0;
  c->trY_new = T;
  (void)Q;
}

// ---------------------------------------------------------------- row norms
// (Y^2)_ii = sum_k Y_ik^2 for symmetric Y, in FP64 on the CUDA cores.  The
// tensor cores accumulate with truncation, which biases sums of positive
// terms (the diagonal of a square) by a relative -K*6e-9; the squaring
// epilogue takes its diagonal from here instead, and the control step gets
// ||Y||_F^2 = sum_i rn_i without that bias.  One warp per row: FP32 FMA over
// 32 consecutive elements (round-to-nearest), FP64 across chunks.
__global__ void __launch_bounds__(256) rownorm_kernel(const float* __restrict__ Y, long long ld_y, long long slot_y,
                                                      const int* __restrict__ Ns, double* __restrict__ rn,
                                                      long long ld_rn, Ctl* __restrict__ ctl,
                                                      double2* __restrict__ partials, unsigned* __restrict__ tickets) {
  const int b = blockIdx.y;
  if (ctl && !ctl[b].next.active) return;
  const int N = Ns[b];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float* Yb = Y + (long long)b * slot_y;
  const bool vec = ((ld_y & 3) == 0) && ((((uintptr_t)Yb) & 15) == 0);
  double blk = 0.0;
  for (int i = blockIdx.x * 8 + warp; i < N; i += gridDim.x * 8) {
    const float* row = Yb + (long long)i * ld_y;
    double acc = 0.0;
    if (vec) {
      const int n4 = N >> 2;
      const float4* r4 = reinterpret_cast<const float4*>(row);
      for (int j0 = 0; j0 < n4; j0 += 32 * 8) {
        float f = 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int j = j0 + u * 32 + lane;
          if (j < n4) {
            const float4 v = __ldcg(r4 + j);
            f = fmaf(v.x, v.x, f);
            f = fmaf(v.y, v.y, f);
            f = fmaf(v.z, v.z, f);
            f = fmaf(v.w, v.w, f);
          }
        }
        acc += (double)f;
      }
      for (int j = (n4 << 2) + lane; j < N; j += 32) acc += (double)row[j] * (double)row[j];
    } else {
      for (int j = lane; j < N; j += 32) acc += (double)row[j] * (double)row[j];
    }
    acc = warp_sum_d(acc);
    if (lane == 0) {
      rn[(long long)b * ld_rn + i] = acc;
      blk += acc;
    }
  }
  if (!ctl) return;
  __shared__ double s_p[8];
  if (lane == 0) s_p[warp] = blk;
  __syncthreads();
  __shared__ bool s_last;
  double2* part = partials + (long long)b * gridDim.x;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += s_p[w];
    part[blockIdx.x] = make_double2(t, 0.0);
    __threadfence();
    s_last = (atomicAdd(&tickets[b], 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;
  __threadfence();
  double Q = 0.0;
  for (unsigned k = 0; k < gridDim.x; ++k) Q += __ldcg(&part[k]).x;
  tickets[b] = 0u;
  Ctl* c = ctl + b;
  control_step(c, c->trY_new, Q);
}

// ---------------------------------------------------------------- split
__global__ void split_kernel(const float* __restrict__ X, long long n, float lo_scale, __half* __restrict__ hi,
                             __half* __restrict__ lo) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    __half h, l;
    split_fp16(X[i], lo_scale, h, l);
    hi[i] = h;
    lo[i] = l;
  }
}

// ---------------------------------------------------------------- split, padded
// X [B][N][ld_x] FP32 -> FP16 planes hi / lo' / hp (each when set) [B][N][ld_h]
// with the row tail [N, ld_h) zeroed.
__device__ __forceinline__ uint32_t pack_half2(__half a, __half b) {
  return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
}

__global__ void split_pad_kernel(const float* __restrict__ X, long long ld_x, long long slot_x, int N, int B,
                                 float lo_scale, __half* __restrict__ hi, __half* __restrict__ lo,
                                 __half* __restrict__ hp, long long ld_h, long long slot_h) {
  const long long rows = (long long)N * B;
  // four elements per thread: float4 loads, 8-byte stores per plane
  const bool vec = ((ld_x | slot_x | ld_h | slot_h) & 3) == 0 && (((uintptr_t)X) & 15) == 0 &&
                   ((((uintptr_t)hi) | ((uintptr_t)lo) | ((uintptr_t)hp)) & 7) == 0;
  for (long long gr = blockIdx.x; gr < rows; gr += gridDim.x) {
    const int b = (int)(gr / N), r = (int)(gr % N);
    const float* xr = X + (long long)b * slot_x + (long long)r * ld_x;
    __half* hr = hi ? hi + (long long)b * slot_h + (long long)r * ld_h : nullptr;
    __half* lr = lo ? lo + (long long)b * slot_h + (long long)r * ld_h : nullptr;
    __half* pr = hp ? hp + (long long)b * slot_h + (long long)r * ld_h : nullptr;
    if (vec) {
      for (int c4 = threadIdx.x; c4 < (int)(ld_h >> 2); c4 += blockDim.x) {
        const int c = c4 << 2;
        float x[4];
        if (c + 4 <= N) {
          const float4 v = reinterpret_cast<const float4*>(xr)[c4];
          x[0] = v.x;
          x[1] = v.y;
          x[2] = v.z;
          x[3] = v.w;
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u) x[u] = (c + u < N) ? xr[c + u] : 0.f;
        }
        __half h[4], l[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) split_fp16(x[u], lo_scale, h[u], l[u]);
        if (hr) *reinterpret_cast<uint2*>(hr + c) = make_uint2(pack_half2(h[0], h[1]), pack_half2(h[2], h[3]));
        if (lr) *reinterpret_cast<uint2*>(lr + c) = make_uint2(pack_half2(l[0], l[1]), pack_half2(l[2], l[3]));
        if (pr) {
          __half q[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) q[u] = __float2half_rn(__half2float(h[u]) * lo_scale);
          *reinterpret_cast<uint2*>(pr + c) = make_uint2(pack_half2(q[0], q[1]), pack_half2(q[2], q[3]));
        }
      }
    } else {
      for (int c = threadIdx.x; c < (int)ld_h; c += blockDim.x) {
        const float x = (c < N) ? xr[c] : 0.f;
        __half h, l;
        split_fp16(x, lo_scale, h, l);
        if (hr) hr[c] = h;
        if (lr) lr[c] = l;
        if (pr) pr[c] = __float2half_rn(__half2float(h) * lo_scale);
      }
    }
  }
}

// ---------------------------------------------------------------- readout
// R[b] = s Y[b] + d[b] I over the N x N block of each slot (diagonal in
// FP64): the input layer's term c_0 X_0 of the finite-temperature readout.
// R must not alias Y (the diagonal is read back after the rows are written).
__global__ void readout_init_kernel(const float* __restrict__ Y, long long ld_y, long long slot_y, int N, float s,
                                    const double* __restrict__ d, float* __restrict__ R) {
  const int b = blockIdx.y;
  const float* Yb = Y + (long long)b * slot_y;
  float* Rb = R + (long long)b * slot_y;
  const bool vec = ((ld_y | slot_y | N) & 3) == 0 && ((((uintptr_t)Y) | ((uintptr_t)R)) & 15) == 0;
  for (int r = blockIdx.x; r < N; r += gridDim.x) {
    const float* yr = Yb + (long long)r * ld_y;
    float* rr = Rb + (long long)r * ld_y;
    if (vec) {
      for (int c4 = threadIdx.x; c4 < (N >> 2); c4 += blockDim.x) {
        const float4 v = reinterpret_cast<const float4*>(yr)[c4];
        reinterpret_cast<float4*>(rr)[c4] = make_float4(s * v.x, s * v.y, s * v.z, s * v.w);
      }
    } else {
      for (int c = threadIdx.x; c < N; c += blockDim.x) rr[c] = s * yr[c];
    }
  }
  // the diagonal of this block's rows in FP64, after the row writes above
  __syncthreads();
  for (long long k = threadIdx.x;; k += blockDim.x) {
    const long long r = blockIdx.x + k * gridDim.x;
    if (r >= N) break;
    Rb[r * ld_y + r] = (float)((double)s * (double)Yb[r * ld_y + r] + d[b]);
  }
}

cudaError_t launch_readout_init(const float* Y, long long ld_y, long long slot_y, int N, int B, float s,
                                const double* d, float* R, int grid_x, cudaStream_t st) {
  dim3 grid(grid_x, B);
  readout_init_kernel<<<grid, 256, 0, st>>>(Y, ld_y, slot_y, N, s, d, R);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- materialise
// out[b] = Y[b] + alpha[b] I (FP64 add on the diagonal, one rounding): the
// full iterate X = alpha I + Y, e.g. for a network checkpoint.  Each block
// copies its rows (float4 when the layout allows) and then sets their
// diagonal: one FP64 operation per row, none per element.
__global__ void materialize_kernel(const float* __restrict__ Y, long long ld_y, long long slot_y, int N,
                                   const double* __restrict__ alpha, float* __restrict__ out, long long ld_o,
                                   long long slot_o) {
  const int b = blockIdx.y;
  const float* Yb = Y + (long long)b * slot_y;
  float* Ob = out + (long long)b * slot_o;
  const bool vec = ((ld_y | slot_y | ld_o | slot_o | N) & 3) == 0 && ((((uintptr_t)Y) | ((uintptr_t)out)) & 15) == 0;
  for (int r = blockIdx.x; r < N; r += gridDim.x) {
    const float* yr = Yb + (long long)r * ld_y;
    float* orow = Ob + (long long)r * ld_o;
    if (vec) {
      for (int c4 = threadIdx.x; c4 < (N >> 2); c4 += blockDim.x)
        reinterpret_cast<float4*>(orow)[c4] = reinterpret_cast<const float4*>(yr)[c4];
    } else {
      for (int c = threadIdx.x; c < N; c += blockDim.x) orow[c] = yr[c];
    }
  }
  // the diagonal of this block's rows in FP64, after the row copies above
  __syncthreads();
  const double a = alpha[b];
  for (long long k = threadIdx.x;; k += blockDim.x) {
    const long long r = blockIdx.x + k * gridDim.x;
    if (r >= N) break;
    Ob[r * ld_o + r] = (float)((double)Yb[r * ld_y + r] + a);
  }
}

// ---------------------------------------------------------------- observable
__global__ void __launch_bounds__(256) observable_kernel(const float* __restrict__ D, const float* __restrict__ A,
                                                         long long n, double* __restrict__ block_out) {
  double acc = 0.0;
  const bool vec = ((((uintptr_t)D) | ((uintptr_t)A)) & 15) == 0;
  if (vec) {
    const long long n4 = n >> 2;
    const float4* D4 = reinterpret_cast<const float4*>(D);
    const float4* A4 = reinterpret_cast<const float4*>(A);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
      const float4 d = __ldcs(D4 + i), a = __ldcs(A4 + i);
      acc += (double)d.x * a.x + (double)d.y * a.y + (double)d.z * a.z + (double)d.w * a.w;
    }
    for (long long i = (n4 << 2) + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
      acc += (double)D[i] * A[i];
  } else {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
      acc += (double)D[i] * A[i];
  }
  acc = warp_sum_d(acc);
  __shared__ double s[8];
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
    block_out[blockIdx.x] = t;
  }
}

// ---------------------------------------------------------------- launchers
cudaError_t launch_gershgorin(const float* H, int N, long long ld, long long slot, int B, double2* partials,
                              unsigned* ticket, Ctl* ctl, double* bounds_out, int grid, cudaStream_t st,
                              long long nan_row) {
  gershgorin_kernel<<<grid, 256, 0, st>>>(H, N, ld, slot, B, partials, ticket, ctl, bounds_out, nan_row);
  return cudaGetLastError();
}

cudaError_t launch_gershgorin_batched(const float* const* Hs, const int* Ns, Ctl* ctl, int batch, double2* partials,
                                     unsigned* tickets, int grid_x, cudaStream_t st) {
  dim3 grid(grid_x, batch);
  gershgorin_batched_kernel<<<grid, 256, 0, st>>>(Hs, Ns, ctl, partials, tickets);
  return cudaGetLastError();
}

cudaError_t launch_input_layer(const float* const* Hs, const int* Ns, long long ld_in, float* Y, long long ld_y,
                               long long slot_y, __half* hi, __half* lo, __half* hp, long long ld_h, long long slot_h,
                               int rows_pad, int cols_pad, float lo_scale, Ctl* ctl, const double* bounds, double2* partials, unsigned* tickets,
                               int shift, int ctl_step, int batch, int grid_x, cudaStream_t st) {
  dim3 grid(grid_x, batch);
  input_layer_kernel<<<grid, 256, 0, st>>>(Hs, Ns, ld_in, Y, ld_y, slot_y, hi, lo, hp, ld_h, slot_h, rows_pad, cols_pad,
                                           lo_scale, ctl,
                                           bounds, partials, tickets, shift, ctl_step);
  return cudaGetLastError();
}

cudaError_t launch_rownorm(const float* Y, long long ld_y, long long slot_y, const int* Ns, int batch, int max_rows,
                           double* rn, long long ld_rn, Ctl* ctl, double2* partials, unsigned* tickets, int grid_x,
                           cudaStream_t st) {
  (void)max_rows;
  dim3 grid(grid_x, batch);
  rownorm_kernel<<<grid, 256, 0, st>>>(Y, ld_y, slot_y, Ns, rn, ld_rn, ctl, partials, tickets);
  return cudaGetLastError();
}

cudaError_t launch_split(const float* X, long long n, float lo_scale, __half* hi, __half* lo, int grid,
                         cudaStream_t st) {
  split_kernel<<<grid, 256, 0, st>>>(X, n, lo_scale, hi, lo);
  return cudaGetLastError();
}

cudaError_t launch_split_pad(const float* X, long long ld_x, long long slot_x, int N, int B, float lo_scale,
                             __half* hi, __half* lo, __half* hp, long long ld_h, long long slot_h, int grid,
                             cudaStream_t st) {
  split_pad_kernel<<<grid, 256, 0, st>>>(X, ld_x, slot_x, N, B, lo_scale, hi, lo, hp, ld_h, slot_h);
  return cudaGetLastError();
}

cudaError_t launch_materialize(const float* Y, long long ld_y, long long slot_y, int N, int B, const double* alpha,
                               float* out, long long ld_o, long long slot_o, int grid_x, cudaStream_t st) {
  dim3 grid(grid_x, B);
  materialize_kernel<<<grid, 256, 0, st>>>(Y, ld_y, slot_y, N, alpha, out, ld_o, slot_o);
  return cudaGetLastError();
}

cudaError_t launch_observable(const float* D, const float* A, long long n, double* block_out, int grid,
                              cudaStream_t st) {
  observable_kernel<<<grid, 256, 0, st>>>(D, A, n, block_out);
  return cudaGetLastError();
}

}  // namespace sp2
