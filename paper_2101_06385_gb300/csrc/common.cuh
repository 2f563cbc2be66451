// Shared device-side definitions of the SP2 library (sm_103a).
//
// The iterate of Alg. 1 is stored as S = alpha I + Y with an FP64 scalar
// alpha kept on the device and Y in FP32 (plus its FP16 planes).  With
// the shift disabled alpha stays 0 and Y = S.  Both branches of the SP2
// layer (Eq. 10 / Alg. 1, W_n = sigma_n I, B_n = (I - W_n) S_{n-1}) and the
// generalised layer of Eq. 16 map onto the same element-wise epilogue
//     Y' = ca * Y + cb * P + cc * I,   P = Y^2 (tensor cores or FFMA),
// with the identity part carried in alpha:
//     S^2 = alpha^2 I + 2 alpha Y + Y^2,
//     sigma = +1: alpha' = alpha^2,            ca = 2 alpha,     cb = +1
//     sigma = -1: alpha' = 2 alpha - alpha^2,  ca = 2 - 2 alpha, cb = -1
// and traces  tr S = N alpha + tr Y,
//             Tr[S^2] = ||S||_F^2 = N alpha^2 + 2 alpha tr Y + ||Y||_F^2.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sp2.h"

namespace sp2 {

constexpr int kMaxL = SP2_MAX_LAYERS;

enum OutMode : int { OUT_Y = 0, OUT_D = 1 };
enum Phase : int { PHASE_LOOP = 0, PHASE_REFINE_A = 1, PHASE_REFINE_B = 2, PHASE_DONE = 3, PHASE_ERROR = 4 };

// Coefficients of one squaring launch.  Written either by the host (network
// and single-layer entry points) or by the device control step (SP2 loop).
// Off-diagonal elements use the FP32 copies; diagonal elements are updated
// in FP64 (exact diagonal of Y^2 from the row norms, exact shifts).
struct LayerParams {
  float ca, cb;       // off-diagonal:  Y'_ij = ca Y_ij + cb P_ij
  int active;         // 0: the launch does nothing (converged / finished)
  int out_mode;       // OutMode
  double ca_d, cb_d;  // diagonal:      Y'_ii = ca_d Y_ii + cb_d P_ii + cc_d
  double cc_d;
  double alpha_out;   // OUT_D: D_ii = Y'_ii + alpha_out, D_ij = Y'_ij
  // readout (finite-temperature expansion, launches with SqArgs::R set):
  // R += rc X' with X' = alpha_new I + Y' (diagonal in FP64); OUT_D writes
  // D = I - R instead of X'
  float rc;
  int pad;
  double rc_d, alpha_new;
};

// Re-centring of the shift: while the spectrum of S is still clustered the
// shift alpha follows the cluster (alpha' = alpha^2 or 2 alpha - alpha^2), so
// Y stays small and FP32 keeps the relative resolution of the HOMO-LUMO gap.
// Once the average lambda (1 - lambda) = IdErr / N falls below this fraction
// the iterate is stored around alpha = 1/2 for good.  S - I/2 of a nearly
// idempotent S squares to nearly I/4, so the off-diagonal sums of Y^2 are
// near zero and the truncating tensor-core accumulation has no preferred
// sign there (it would otherwise shrink them and bias the final trace).
constexpr double kRecenterFrac = 0.01;

// Device-resident state of one SP2 solve (Alg. 1 scalars, FP64).
struct Ctl {
  // configuration
  int N, max_iter, n_occ, shift;
  double tol, eps;
  // state
  int phase, n, stop_pending, converged_by;
  int status, sigma_a, recentered, pad1;
  double alpha, alpha_next;   // shift of the stored iterate / of the one being computed
  double trY, sqY;            // tr Y, ||Y||_F^2 of the stored Y
  double trY_new;             // tr Y of the iterate just written (set by the squaring launch)
  double e_min, e_max;
  double trace_final;
  LayerParams next;           // parameters of the next squaring launch
  int sigma[kMaxL + 1];       // sigma[k] = sigma_k, sigma[0] = 0
  double iderr[kMaxL + 1];    // iderr[k] = IdErr_k
  // accelerated solve (Sec. "Accelerated Deep-NN SP2")
  int accel, pad2;
  double acc_homo, acc_lumo;  // caller's HOMO / LUMO energy estimates
  double acc_l, acc_h;        // unoccupied eigenvalues of the scaled iterate in [0, l], occupied in [h, 1]
};

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ void split_fp16(float x, float lo_scale, __half& hi, __half& lo) {
  // Eq. 12: hi = FP16[x], lo = FP16[2^s (x - hi)]; x - hi is exact in FP32.
  hi = __float2half_rn(x);
  lo = __float2half_rn((x - __half2float(hi)) * lo_scale);
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Branch sigma applied to the stored iterate: sets alpha_next and the launch
// coefficients (see the header comment).  After re-centring, the new iterate
// is stored around alpha = 1/2: the shift difference goes into cc.
__device__ inline void set_branch(Ctl* c, int sigma, bool final_layer) {
  const double a = c->alpha;
  double an, ca, cb, cc = 0.0;
  if (sigma > 0) {
    an = a * a;
    ca = 2.0 * a;
    cb = 1.0;
  } else {
    an = 2.0 * a - a * a;
    ca = 2.0 - 2.0 * a;
    cb = -1.0;
  }
  if (c->recentered) {
    cc = an - 0.5;
    an = 0.5;
  }
  c->alpha_next = an;
  LayerParams p;
  p.ca = (float)ca;
  p.cb = (float)cb;
  p.ca_d = ca;
  p.cb_d = cb;
  p.cc_d = cc;
  p.alpha_out = final_layer ? an : 0.0;
  p.active = 1;
  p.out_mode = final_layer ? OUT_D : OUT_Y;
  p.rc = 0.f;
  p.pad = 0;
  p.rc_d = 0.0;
  p.alpha_new = 0.0;
  c->next = p;
}

// Control step of Alg. 1, run by one thread after the launch that stored a
// new iterate (the input layer for n = 0).  trY / sqY are the FP64 sums of
// the Y just stored.  Decides sigma_{n+1}, IdErr_{n+1} and the stop rules
// (IdErr <= tol, IdErr <= 0, the 4.5 rule after a sign change, max_iter), or
// moves on to the two refinement layers of Eq. 15.
// Generalised layer S' = a S^2 + b S + c I on the stored S = alpha I + Y:
// S' = (a alpha^2 + b alpha + c) I + (2 a alpha + b) Y + a Y^2.
__device__ inline void set_poly(Ctl* c, double a, double b, double cp, bool final_layer) {
  const double al = c->alpha;
  double an = a * al * al + b * al + cp;
  const double ca = 2.0 * a * al + b, cb = a;
  double cc = 0.0;
  if (c->recentered) {
    cc = an - 0.5;
    an = 0.5;
  } else if (!c->shift) {
    cc = an;
    an = 0.0;
  }
  c->alpha_next = an;
  LayerParams p;
  p.ca = (float)ca;
  p.cb = (float)cb;
  p.ca_d = ca;
  p.cb_d = cb;
  p.cc_d = cc;
  p.alpha_out = final_layer ? an : 0.0;
  p.active = 1;
  p.out_mode = final_layer ? OUT_D : OUT_Y;
  p.rc = 0.f;
  p.pad = 0;
  p.rc_d = 0.0;
  p.alpha_new = 0.0;
  c->next = p;
}

// Layer of the accelerated scheme on bounds (l, h): shift and rescale so the
// side farther from its fixed point folds onto itself, then square.
//   1 - h <= l: p(x) = ((x - s)/(1 - s))^2, s = l/2   (0 and l meet at p = (s/(1-s))^2)
//   otherwise:  q(x) = 1 - ((1 - x - t)/(1 - t))^2, t = (1 - h)/2
__device__ inline int accel_layer(double& l, double& h, double& a, double& b, double& cp) {
  if (1.0 - h <= l) {
    const double s = 0.5 * l, d = 1.0 - s;
    a = 1.0 / (d * d);
    b = -2.0 * s / (d * d);
    cp = s * s / (d * d);
    const double hs = (h - s) / d;
    l = (s / d) * (s / d);
    h = hs * hs;
    return 1;
  }
  const double t = 0.5 * (1.0 - h), d = 1.0 - t;
  a = -1.0 / (d * d);
  b = 2.0 / d;
  cp = 0.0;
  const double lt = (1.0 - l - t) / d;
  h = 1.0 - (t / d) * (t / d);
  l = 1.0 - lt * lt;
  return -1;
}

// Control step of the accelerated solve: the layers follow the bounds alone;
// IdErr is recorded for the statistics and the re-centring of the shift.
__device__ inline void accel_control_step(Ctl* c, double trY, double sqY) {
  const double N = (double)c->N;
  if (c->phase == PHASE_LOOP) {
    const int n1 = c->n + 1;
    const double a = c->alpha;
    const double err = N * a * (1.0 - a) + (1.0 - 2.0 * a) * trY - sqY;
    if (c->n == 0) {
      const double w = c->e_max - c->e_min;
      c->acc_l = fmin(fmax((c->e_max - c->acc_lumo) / w, 0.0), 1.0);
      c->acc_h = fmin(fmax((c->e_max - c->acc_homo) / w, 0.0), 1.0);
      if (!(c->acc_l < c->acc_h)) {
        c->status = SP2_ERR_INVALID_ARG;
        c->phase = PHASE_ERROR;
        c->next.active = 0;
        return;
      }
    }
    c->iderr[n1] = err;
    if (c->shift && !c->recentered && err <= kRecenterFrac * N) c->recentered = 1;
    double l = c->acc_l, h = c->acc_h, pa, pb, pc;
    const int s = accel_layer(l, h, pa, pb, pc);
    c->acc_l = l;
    c->acc_h = h;
    c->sigma[n1] = s;
    c->n = n1;
    const bool done = fmax(l, 1.0 - h) <= c->tol;
    const bool final_layer = done || n1 >= c->max_iter;
    if (final_layer) {
      c->converged_by = done ? SP2_STOP_BOUNDS : SP2_STOP_MAXITER;
      c->phase = PHASE_REFINE_B;  // the next step (after the OUT_D launch) finishes
    }
    set_poly(c, pa, pb, pc, final_layer);
  } else if (c->phase == PHASE_REFINE_B) {
    c->trace_final = N * c->alpha + trY;
    c->phase = PHASE_DONE;
    c->next.active = 0;
    if (c->status == SP2_OK && c->converged_by == SP2_STOP_MAXITER) c->status = SP2_NOT_CONVERGED;
  }
}

__device__ inline void control_step(Ctl* c, double trY, double sqY) {
  c->trY = trY;
  c->sqY = sqY;
  c->alpha = c->alpha_next;
  if (c->accel) {
    accel_control_step(c, trY, sqY);
    return;
  }
  const double N = (double)c->N;
  if (c->phase == PHASE_LOOP) {
    if (c->stop_pending) {
      int s = (c->n >= 3) ? c->sigma[c->n - 2] : 1;  // f_final order from sigma_{n-2}
      s = (s >= 0) ? 1 : -1;
      c->sigma_a = s;
      c->phase = PHASE_REFINE_A;
      set_branch(c, s, false);
      return;
    }
    const int n1 = c->n + 1;
    const double a = c->alpha;
    const double NS = N * a + trY;                      // Tr[S_n]
    const double NX = N * a * a + 2.0 * a * trY + sqY;  // Tr[S_n^2] = ||S_n||_F^2
    const double err = N * a * (1.0 - a) + (1.0 - 2.0 * a) * trY - sqY;  // N_S - N_X
    const double no = (double)c->n_occ;
    const double v = fabs(2.0 * NS - NX - no) - fabs(NX - no) - (double)c->sigma[c->n] * c->eps;
    const int s = (v >= 0.0) ? 1 : -1;
    c->sigma[n1] = s;
    c->iderr[n1] = err;
    if (c->shift && !c->recentered && err <= kRecenterFrac * N) c->recentered = 1;
    int stop = SP2_STOP_NONE;
    if (c->tol > 0.0 && err <= c->tol)
      stop = SP2_STOP_TOL;
    else if (err <= 0.0)
      stop = SP2_STOP_IDERR;
    else if (n1 > 2 && c->sigma[n1 - 1] != c->sigma[n1 - 2] && err > 4.5 * c->iderr[n1 - 2] * c->iderr[n1 - 2])
      stop = SP2_STOP_RULE45;
    else if (n1 >= c->max_iter)
      stop = SP2_STOP_MAXITER;
    c->n = n1;
    c->stop_pending = stop;
    if (stop) c->converged_by = stop;
    set_branch(c, s, false);
  } else if (c->phase == PHASE_REFINE_A) {
    c->phase = PHASE_REFINE_B;
    set_branch(c, -c->sigma_a, true);
  } else if (c->phase == PHASE_REFINE_B) {
    c->trace_final = N * c->alpha + trY;
    c->phase = PHASE_DONE;
    c->next.active = 0;
    if (c->status == SP2_OK && c->converged_by == SP2_STOP_MAXITER) c->status = SP2_NOT_CONVERGED;
  }
}

// Tile descriptor of the squaring kernels: instance b, block row I, block
// column J (I <= J in units of the kernel's tile), and sub-row h.
__host__ __device__ inline uint32_t pack_tile(int b, int I, int J, int h) {
  return ((uint32_t)b << 20) | ((uint32_t)I << 11) | ((uint32_t)J << 2) | (uint32_t)h;
}
__host__ __device__ inline void unpack_tile(uint32_t t, int& b, int& I, int& J, int& h) {
  b = (int)(t >> 20);
  I = (int)((t >> 11) & 0x1FF);
  J = (int)((t >> 2) & 0x1FF);
  h = (int)(t & 3);
}

}  // namespace sp2
