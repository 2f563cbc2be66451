// FP32 squaring on the CUDA cores (FFMA): the paper's "GPU-only" comparator
// (Sec. 4, tensor cores disabled), with the same fused layer epilogue as the
// tensor-core kernel.  Upper 128 x 128 tiles of P = Y Y (Y symmetric, so
// both operands are row panels); diagonal tiles are computed in full, off-
// diagonal tiles are stored twice (mirrored).
#include "common.cuh"
#include "kernels.h"
#include "tile_finish.cuh"

namespace sp2 {

namespace {
constexpr int BM = kSimtB;
constexpr int BK = 8;
constexpr int PADM = BM + 4;

__device__ __forceinline__ float4 load4_masked(const float* __restrict__ Y, long long ld, int N, int r, int k,
                                              bool vec_ok) {
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (r >= N) return v;
  const float* p = Y + (long long)r * ld + k;
  if (vec_ok && k + 3 < N) return __ldg(reinterpret_cast<const float4*>(p));
  if (k + 3 < N) return make_float4(p[0], p[1], p[2], p[3]);
  if (k < N) v.x = p[0];
  if (k + 1 < N) v.y = p[1];
  if (k + 2 < N) v.z = p[2];
  return v;
}
}  // namespace

__global__ void __launch_bounds__(256) syrk_simt_kernel(const SqArgs a) {
  __shared__ __align__(16) float As[2][BK][PADM];
  __shared__ __align__(16) float Bs[2][BK][PADM];
  __shared__ LayerParams s_p;
  __shared__ double s_red[8][2];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int lr = tid >> 1, lk = (tid & 1) * 4;

  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    int b, I, J, h;
    unpack_tile(a.tiles[t], b, I, J, h);
    if (tid == 0) s_p = a.ctl ? a.ctl[b].next : a.lp[a.lp_per_instance ? b : 0];
    __syncthreads();
    const LayerParams p = s_p;
    __syncthreads();
    if (!p.active) continue;
    const int N = a.Ns[b];
    const long long ld = a.ld_y;
    const float* Y = a.Yin + (long long)b * a.slot_y;
    const bool vec_ok = ((ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(Y) & 15) == 0);
    const int r0 = I * BM, c0 = J * BM;

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    float4 ra = load4_masked(Y, ld, N, r0 + lr, lk, vec_ok);
    float4 rb = load4_masked(Y, ld, N, c0 + lr, lk, vec_ok);
    As[0][lk + 0][lr] = ra.x; As[0][lk + 1][lr] = ra.y; As[0][lk + 2][lr] = ra.z; As[0][lk + 3][lr] = ra.w;
    Bs[0][lk + 0][lr] = rb.x; Bs[0][lk + 1][lr] = rb.y; Bs[0][lk + 2][lr] = rb.z; Bs[0][lk + 3][lr] = rb.w;
    __syncthreads();
    const int nk = (N + BK - 1) / BK;
    for (int kb = 0; kb < nk; ++kb) {
      const int cur = kb & 1;
      if (kb + 1 < nk) {
        ra = load4_masked(Y, ld, N, r0 + lr, (kb + 1) * BK + lk, vec_ok);
        rb = load4_masked(Y, ld, N, c0 + lr, (kb + 1) * BK + lk, vec_ok);
      }
#pragma unroll
      for (int k = 0; k < BK; ++k) {
        const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][k][ty * 4]);
        const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][k][64 + ty * 4]);
        const float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][k][tx * 4]);
        const float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][k][64 + tx * 4]);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
      }
      if (kb + 1 < nk) {
        const int nx = cur ^ 1;
        As[nx][lk + 0][lr] = ra.x; As[nx][lk + 1][lr] = ra.y; As[nx][lk + 2][lr] = ra.z; As[nx][lk + 3][lr] = ra.w;
        Bs[nx][lk + 0][lr] = rb.x; Bs[nx][lk + 1][lr] = rb.y; Bs[nx][lk + 2][lr] = rb.z; Bs[nx][lk + 3][lr] = rb.w;
      }
      __syncthreads();
    }

    // fused layer epilogue: Y' = ca Y + cb P + cc I, mirrored store, partials
    const bool mirror = (I != J);
    const bool outD = (p.out_mode == OUT_D);
    float* Yo = a.Yout + (long long)b * a.slot_y;
    float* D = outD ? a.Dptr[b] : nullptr;
    double tr = 0.0;
    float sqf = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = r0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
      if (r >= N) continue;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = c0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
        if (c >= N) continue;
        const float yold = Y[(long long)r * ld + c];
        float y, d;
        if (r == c) {
          const double pd = a.rn ? a.rn[(long long)b * a.ld_rn + r] : (double)acc[i][j];
          const double yd = p.ca_d * (double)yold + p.cb_d * pd + p.cc_d;
          tr += yd;
          y = (float)yd;
          d = (float)(yd + p.alpha_out);
        } else {
          y = fmaf(p.ca, yold, p.cb * acc[i][j]);
          d = y;
        }
        sqf = fmaf(y, y, sqf);
        if (outD) {
          D[(long long)r * N + c] = d;
          if (mirror) D[(long long)c * N + r] = d;
        } else {
          Yo[(long long)r * ld + c] = y;
          if (mirror) Yo[(long long)c * ld + r] = y;
        }
      }
    }
    double sq = (double)sqf * (mirror ? 2.0 : 1.0);
    tr = warp_sum_d(tr);
    sq = warp_sum_d(sq);
    if ((tid & 31) == 0) {
      s_red[tid >> 5][0] = tr;
      s_red[tid >> 5][1] = sq;
    }
    __syncthreads();
    if (tid < 32) {
      double T = 0.0, Q = 0.0;
      if (tid == 0)
        for (int w = 0; w < 8; ++w) {
          T += s_red[w][0];
          Q += s_red[w][1];
        }
      finish_tile_warp(a, t, b, T, Q, p.out_mode);
    }
    __syncthreads();
  }
}

cudaError_t launch_syrk_simt(const SqArgs& a, int grid, cudaStream_t st) {
  syrk_simt_kernel<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace sp2
