// Residual of a refinement sweep as a streaming stencil: r = f - L_h(Phi + Plo) (Eq. poi), written
// as a float field for the forward transform that follows, plus sum r^2.
//
// A thread owns one (i, j) column and marches along z through a chunk of planes, keeping Phi at
// k-1, k and k+1 in registers (the z neighbours cost no load); the x and y neighbours of plane k
// are the values the neighbouring threads loaded one step earlier, so they come from L1.  Each
// point costs two DRAM reads (f and the next Phi) and one write.  The arithmetic is that of the
// fused x-pass (double-float Phi part, float Plo part).
#include <algorithm>

#include "plan.cuh"
#include "stencil.cuh"

namespace cans {
namespace {

constexpr int RX = 32, RY = 8;  // CTA tile of columns

template <bool PLO>
__global__ void __launch_bounds__(RX * RY) res_kernel(const double* __restrict__ f, const float* __restrict__ Phi,
                                                      const float* __restrict__ Plo, float* __restrict__ r,
                                                      StencilDF S, int kchunk, double* norm_acc) {
  const int nx = S.n[0], ny = S.n[1], nz = S.n[2];
  const int i = blockIdx.x * RX + threadIdx.x, j = blockIdx.y * RY + threadIdx.y;
  const bool active = i < nx && j < ny;
  float acc = 0.f;
  if (active) {
    const size_t sz = (size_t)nx * ny;
    const bool wx = S.bc[0] != BC_P, wy = S.bc[1] != BC_P, wz = S.bc[2] != BC_P;
    const int im = (i == 0) ? nx - 1 : i - 1, ip = (i == nx - 1) ? 0 : i + 1;
    const int jm = (j == 0) ? ny - 1 : j - 1, jp = (j == ny - 1) ? 0 : j + 1;
    const bool gxm = wx && i == 0, gxp = wx && i == nx - 1, gym = wy && j == 0, gyp = wy && j == ny - 1;
    const size_t c0 = (size_t)j * nx + i;
    const size_t cxm = (size_t)j * nx + im, cxp = (size_t)j * nx + ip;
    const size_t cym = (size_t)jm * nx + i, cyp = (size_t)jp * nx + i;
    const int k0 = blockIdx.z * kchunk, k1 = min(nz, k0 + kchunk);
    // Phi (and Plo) at k0 - 1 (periodic wrap; a wall ghost is formed at k = 0 below)
    const size_t kprev = (k0 == 0) ? (size_t)(nz - 1) : (size_t)(k0 - 1);
    float p_prev = Phi[kprev * sz + c0], p_cur = Phi[(size_t)k0 * sz + c0];
    float q_prev = 0.f, q_cur = 0.f;
    if (PLO) {
      q_prev = Plo[kprev * sz + c0];
      q_cur = Plo[(size_t)k0 * sz + c0];
    }
    for (int k = k0; k < k1; ++k) {
      const size_t o = (size_t)k * sz;
      const size_t on = (k == nz - 1) ? 0 : o + sz;  // plane k+1 (periodic wrap)
      const float p_next = Phi[on + c0];
      const float xm = gxm ? wall_ghost(S.bc[0], p_cur) : Phi[o + cxm];
      const float xp = gxp ? wall_ghost(S.bc[0], p_cur) : Phi[o + cxp];
      const float ym = gym ? wall_ghost(S.bc[1], p_cur) : Phi[o + cym];
      const float yp = gyp ? wall_ghost(S.bc[1], p_cur) : Phi[o + cyp];
      const float zm = (wz && k == 0) ? wall_ghost(S.bc[2], p_cur) : p_prev;
      const float zp = (wz && k == nz - 1) ? wall_ghost(S.bc[2], p_cur) : p_next;
      df a = df_split(f[o + c0]);
      if (S.iso) {
        const df sx = two_sum(xm, xp);
        const df sy = two_sum(ym, yp);
        const df s2 = two_sum(sx.hi, sy.hi);
        const df d = two_sum(s2.hi, -4.f * p_cur);
        a = df_sub_prod(a, S.idx2, df_make(d.hi, __fadd_rn(d.lo, __fadd_rn(s2.lo, __fadd_rn(sx.lo, sy.lo)))));
      } else {
        a = df_sub_prod(a, S.idx2, second_difference(xm, xp, p_cur));
        a = df_sub_prod(a, S.idy2, second_difference(ym, yp, p_cur));
      }
      a = df_sub_prod(a, df_make(S.sc_hi[k], S.sc_lo[k]), two_sum(zp, -p_cur));
      a = df_sub_prod(a, df_make(S.sa_hi[k], S.sa_lo[k]), two_sum(zm, -p_cur));
      float rr = a.hi + a.lo;
      if (PLO) {
        const float q_next = Plo[on + c0];
        const float qxm = gxm ? wall_ghost(S.bc[0], q_cur) : Plo[o + cxm];
        const float qxp = gxp ? wall_ghost(S.bc[0], q_cur) : Plo[o + cxp];
        const float qym = gym ? wall_ghost(S.bc[1], q_cur) : Plo[o + cym];
        const float qyp = gyp ? wall_ghost(S.bc[1], q_cur) : Plo[o + cyp];
        const float qzm = (wz && k == 0) ? wall_ghost(S.bc[2], q_cur) : q_prev;
        const float qzp = (wz && k == nz - 1) ? wall_ghost(S.bc[2], q_cur) : q_next;
        rr -= S.idx2.hi * (qxm + qxp - 2.f * q_cur) + S.idy2.hi * (qym + qyp - 2.f * q_cur) +
              S.sc_hi[k] * (qzp - q_cur) + S.sa_hi[k] * (qzm - q_cur);
        q_prev = q_cur;
        q_cur = q_next;
      }
      r[o + c0] = rr;
      acc = __fmaf_rn(rr, rr, acc);
      p_prev = p_cur;
      p_cur = p_next;
    }
  }
  if (norm_acc != nullptr) {
    __shared__ float red[RX * RY / 32];
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
    const int t = threadIdx.y * RX + threadIdx.x;
    if ((t & 31) == 0) red[t >> 5] = acc;
    __syncthreads();
    if (t == 0) {
      float s = 0.f;
      for (int w = 0; w < RX * RY / 32; ++w) s += red[w];
      atomicAdd(norm_acc, (double)s);
    }
  }
}

}  // namespace

cudaError_t launch_residual(const cans_plan_s* P, const double* f, const float* Phi, const float* Plo, bool plo,
                            float* r, double* norm_acc, cudaStream_t st) {
  const int nx = P->n[0], ny = P->n[1], nz = P->n[2];
  const int kchunk = std::min(nz, 64);
  dim3 grid((nx + RX - 1) / RX, (ny + RY - 1) / RY, (nz + kchunk - 1) / kchunk);
  dim3 block(RX, RY);
  const StencilDF S = stencil_df(P);
  if (plo)
    res_kernel<true><<<grid, block, 0, st>>>(f, Phi, Plo, r, S, kchunk, norm_acc);
  else
    res_kernel<false><<<grid, block, 0, st>>>(f, Phi, Plo, r, S, kchunk, norm_acc);
  return cudaGetLastError();
}

}  // namespace cans
