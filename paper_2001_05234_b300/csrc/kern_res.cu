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

// coef * x as a double-float (coef and x double-float): the product's exact head and a float tail
__device__ __forceinline__ df df_prod(df coef, df x) {
  df p = two_prod(coef.hi, x.hi);
  p.lo = __fmaf_rn(coef.hi, x.lo, __fmaf_rn(coef.lo, x.hi, p.lo));
  return p;
}
// acc + coef * x
__device__ __forceinline__ df df_add_prod(df acc, df coef, df x) {
  const df p = df_prod(coef, x);
  const df s = two_sum(acc.hi, p.hi);
  return df_make(s.hi, __fadd_rn(s.lo, __fadd_rn(acc.lo, p.lo)));
}

// PM bit 0: Plo is nonzero (later sweeps); bit 1: the Helmholtz shift term (kept out of the Poisson
// instantiations' inner loop)
template <int PM, int BX, int BY, int BZ>
__global__ void __launch_bounds__(RX * RY, 4) res_kernel(const double* __restrict__ f, const float* __restrict__ Phi,
                                                      const float* __restrict__ Plo, float* __restrict__ r,
                                                      StencilDF S, int kchunk, double* norm_acc) {
  constexpr bool PLO = (PM & 1) != 0, SHIFT = (PM & 2) != 0;
  __shared__ float4 zc[64];  // (c_k hi, c_k lo, a_k hi, a_k lo) of the chunk's planes
  const int nx = S.n[0], ny = S.n[1], nz = S.n[2];
  const int k0 = blockIdx.z * kchunk, k1 = min(nz, k0 + kchunk);
  for (int q = threadIdx.y * RX + threadIdx.x; q < k1 - k0; q += RX * RY)
    zc[q] = make_float4(S.sc_hi[k0 + q], S.sc_lo[k0 + q], S.sa_hi[k0 + q], S.sa_lo[k0 + q]);
  __syncthreads();
  const int i = blockIdx.x * RX + threadIdx.x, j = blockIdx.y * RY + threadIdx.y;
  const bool active = i < nx && j < ny;
  float acc = 0.f;
  if (active) {
    const int sz = nx * ny;  // in-plane offsets stay 32-bit (a plane has < 2^31 points)
    const int im = (i == 0) ? nx - 1 : i - 1, ip = (i == nx - 1) ? 0 : i + 1;
    const int jm = (j == 0) ? ny - 1 : j - 1, jp = (j == ny - 1) ? 0 : j + 1;
    const bool gxm = BX != BC_P && i == 0, gxp = BX != BC_P && i == nx - 1;
    const bool gym = BY != BC_P && j == 0, gyp = BY != BC_P && j == ny - 1;
    // x / y wall ghosts: the sign of each wall (compile time for NN / DD, from S for a mixed pair, BC_ND)
    const float sxm = (BX == BC_NN) ? 1.f : (BX == BC_DD) ? -1.f : ((S.xlo == BC_NN) ? 1.f : -1.f);
    const float sxp = (BX == BC_NN) ? 1.f : (BX == BC_DD) ? -1.f : ((S.xhi == BC_NN) ? 1.f : -1.f);
    const float sym = (BY == BC_NN) ? 1.f : (BY == BC_DD) ? -1.f : ((S.ylo == BC_NN) ? 1.f : -1.f);
    const float syp = (BY == BC_NN) ? 1.f : (BY == BC_DD) ? -1.f : ((S.yhi == BC_NN) ? 1.f : -1.f);
    const int c0 = j * nx + i;
    const int dxm = j * nx + im - c0, dxp = j * nx + ip - c0, dym = jm * nx + i - c0, dyp = jp * nx + i - c0;
    const int kprev = (k0 == 0) ? nz - 1 : k0 - 1;
    const float* pp = Phi + (size_t)k0 * sz + c0;  // Phi at (i, j, k)
    const double* fp = f + (size_t)k0 * sz + c0;
    float* rp = r + (size_t)k0 * sz + c0;
    const float p_first_prev = Phi[(size_t)kprev * sz + c0];
    float p_cur = pp[0];
    // Phi_{k-1} - Phi_k exactly (k = k0; a wall ghost at k = 0)
    // z wall ghosts: Neumann mirrors, Dirichlet negates; BZ = NN / DD fix both walls at compile time,
    // BZ = BC_ND takes each wall's own rule from S (the mixed pairs)
    const float zsl = (BZ == BC_NN) ? 1.f : (BZ == BC_DD) ? -1.f : ((S.zlo == BC_NN) ? 1.f : -1.f);
    const float zsh = (BZ == BC_NN) ? 1.f : (BZ == BC_DD) ? -1.f : ((S.zhi == BC_NN) ? 1.f : -1.f);
    df dm = two_sum((BZ != BC_P && k0 == 0) ? zsl * p_cur : p_first_prev, -p_cur);
    const float* qp = PLO ? Plo + (size_t)k0 * sz + c0 : nullptr;
    float q_prev = 0.f, q_cur = 0.f;
    if (PLO) {
      q_prev = Plo[(size_t)kprev * sz + c0];
      q_cur = qp[0];
    }
    // register ring of the next PF planes' f and Phi_{k+1}: the loads of plane k + PF are issued
    // while plane k is computed, so each thread keeps PF plane loads in flight
    constexpr int PF = 4;
    double fr[PF];
    float pr[PF];
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      const int k = k0 + u;
      if (k < k1) {
        fr[u] = fp[(size_t)u * sz];
        pr[u] = (k == nz - 1) ? Phi[c0] : pp[(size_t)(u + 1) * sz];  // Phi_{k+1}, periodic wrap
      }
    }
    // the x / y neighbours of the next plane, loaded one plane ahead of their use
    float nxm = pp[dxm], nxp = pp[dxp], nym = pp[dym], nyp = pp[dyp];
    for (int kb = k0; kb < k1; kb += PF) {
#pragma unroll
      for (int u = 0; u < PF; ++u) {
        const int k = kb + u;
        if (k < k1) {
          const bool top = (k == nz - 1);
          const float p_next = pr[u];
          const double fk = fr[u];
          if (k + PF < k1) {  // refill this ring slot with plane k + PF
            fr[u] = fp[(size_t)PF * sz];
            pr[u] = (k + PF == nz - 1) ? Phi[c0] : pp[(size_t)(PF + 1) * sz];
          }
          const float xm = gxm ? sxm * p_cur : nxm;
          const float xp = gxp ? sxp * p_cur : nxp;
          const float ym = gym ? sym * p_cur : nym;
          const float yp = gyp ? syp * p_cur : nyp;
          if (k + 1 < k1) {
            nxm = pp[sz + dxm];
            nxp = pp[sz + dxp];
            nym = pp[sz + dym];
            nyp = pp[sz + dyp];
          }
          const float zp = (BZ != BC_P && top) ? zsh * p_cur : p_next;
          const df dp = two_sum(zp, -p_cur);  // Phi_{k+1} - Phi_k exactly
          const float4 co = zc[k - k0];
          // L_h Phi as a double-float
          df L;
          if (S.iso) {
            const df sx = two_sum(xm, xp);
            const df sy = two_sum(ym, yp);
            const df s2 = two_sum(sx.hi, sy.hi);
            const df d = two_sum(s2.hi, -4.f * p_cur);
            L = df_prod(S.idx2, df_make(d.hi, __fadd_rn(d.lo, __fadd_rn(s2.lo, __fadd_rn(sx.lo, sy.lo)))));
          } else {
            L = df_prod(S.idx2, second_difference(xm, xp, p_cur));
            L = df_add_prod(L, S.idy2, second_difference(ym, yp, p_cur));
          }
          L = df_add_prod(L, df_make(co.x, co.y), dp);
          L = df_add_prod(L, df_make(co.z, co.w), dm);
          if (SHIFT) L = df_add_prod(L, S.shift, df_make(p_cur, 0.f));
          // r = (f_hi - L_hi) + (f_lo - L_lo): the first difference is exact when r is small against
          // f (Sterbenz), and otherwise rounds relative to r itself
          const df fs = df_split_rz(fk);
          float rr = __fadd_rn(__fsub_rn(fs.hi, L.hi), __fsub_rn(fs.lo, L.lo));
          if (PLO) {
            const long long dzp = top ? -(long long)(nz - 1) * sz : (long long)sz;
            const float q_next = qp[dzp];
            const float qxm = gxm ? sxm * q_cur : qp[dxm];
            const float qxp = gxp ? sxp * q_cur : qp[dxp];
            const float qym = gym ? sym * q_cur : qp[dym];
            const float qyp = gyp ? syp * q_cur : qp[dyp];
            const float qzm = (BZ != BC_P && k == 0) ? zsl * q_cur : q_prev;
            const float qzp = (BZ != BC_P && top) ? zsh * q_cur : q_next;
            rr -= S.idx2.hi * (qxm + qxp - 2.f * q_cur) + S.idy2.hi * (qym + qyp - 2.f * q_cur) +
                  co.x * (qzp - q_cur) + co.z * (qzm - q_cur) + (SHIFT ? S.shift.hi * q_cur : 0.f);
            q_prev = q_cur;
            q_cur = q_next;
            qp += sz;
          }
          *rp = rr;
          acc = __fmaf_rn(rr, rr, acc);
          // next plane: Phi_k - Phi_{k+1} = -(Phi_{k+1} - Phi_k) exactly (TwoSum is odd and symmetric)
          dm = df_make(-dp.hi, -dp.lo);
          p_cur = p_next;
          pp += sz;
          fp += sz;
          rp += sz;
        }
      }
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

// The same stencil with two x-neighbouring points per thread (nx even, f 16-byte and the float
// fields 8-byte aligned): f, Phi_{k+1}, the y neighbours and r move as 8- or 16-byte vectors, the
// inner x neighbours of the pair are each other's centre values, and the address and loop work is
// shared by the two points.  Same arithmetic per point as res_kernel.
constexpr int R2X = 32, R2Y = 8;  // threads of a CTA; a thread owns points i, i + 1

template <int PM, int BX, int BY, int BZ>
__global__ void __launch_bounds__(R2X * R2Y, 3) res2_kernel(const double* __restrict__ f, const float* __restrict__ Phi,
                                                         const float* __restrict__ Plo, float* __restrict__ r,
                                                         StencilDF S, int kchunk, double* norm_acc) {
  constexpr bool PLO = (PM & 1) != 0, SHIFT = (PM & 2) != 0;
  __shared__ float4 zc[64];  // (c_k hi, c_k lo, a_k hi, a_k lo) of the chunk's planes
  const int nx = S.n[0], ny = S.n[1], nz = S.n[2];
  const int k0 = blockIdx.z * kchunk, k1 = min(nz, k0 + kchunk);
  for (int q = threadIdx.y * R2X + threadIdx.x; q < k1 - k0; q += R2X * R2Y)
    zc[q] = make_float4(S.sc_hi[k0 + q], S.sc_lo[k0 + q], S.sa_hi[k0 + q], S.sa_lo[k0 + q]);
  __syncthreads();
  const int i = 2 * (blockIdx.x * R2X + threadIdx.x), j = blockIdx.y * R2Y + threadIdx.y;
  float acc = 0.f;
  if (i < nx && j < ny) {  // nx is even, so i + 1 < nx as well
    const int sz = nx * ny;
    const int im = (i == 0) ? nx - 1 : i - 1, ip = (i + 2 == nx) ? 0 : i + 2;  // outer x neighbours
    const int jm = (j == 0) ? ny - 1 : j - 1, jp = (j == ny - 1) ? 0 : j + 1;
    const bool gxm = BX != BC_P && i == 0, gxp = BX != BC_P && i + 2 == nx;
    const bool gym = BY != BC_P && j == 0, gyp = BY != BC_P && j == ny - 1;
    const float sxm = (BX == BC_NN) ? 1.f : (BX == BC_DD) ? -1.f : ((S.xlo == BC_NN) ? 1.f : -1.f);
    const float sxp = (BX == BC_NN) ? 1.f : (BX == BC_DD) ? -1.f : ((S.xhi == BC_NN) ? 1.f : -1.f);
    const float sym = (BY == BC_NN) ? 1.f : (BY == BC_DD) ? -1.f : ((S.ylo == BC_NN) ? 1.f : -1.f);
    const float syp = (BY == BC_NN) ? 1.f : (BY == BC_DD) ? -1.f : ((S.yhi == BC_NN) ? 1.f : -1.f);
    const float zsl = (BZ == BC_NN) ? 1.f : (BZ == BC_DD) ? -1.f : ((S.zlo == BC_NN) ? 1.f : -1.f);
    const float zsh = (BZ == BC_NN) ? 1.f : (BZ == BC_DD) ? -1.f : ((S.zhi == BC_NN) ? 1.f : -1.f);
    const int c0 = j * nx + i;
    const int dxm = j * nx + im - c0, dxp = j * nx + ip - c0, dym = jm * nx + i - c0, dyp = jp * nx + i - c0;
    const int kprev = (k0 == 0) ? nz - 1 : k0 - 1;
    const float* pp = Phi + (size_t)k0 * sz + c0;
    const double* fp = f + (size_t)k0 * sz + c0;
    float* rp = r + (size_t)k0 * sz + c0;
    auto ld2 = [](const float* a) { return *reinterpret_cast<const float2*>(a); };
    float2 p_cur = ld2(pp);
    const float2 pprev = ld2(Phi + (size_t)kprev * sz + c0);
    const bool zwall0 = BZ != BC_P && k0 == 0;
    df dm0 = two_sum(zwall0 ? zsl * p_cur.x : pprev.x, -p_cur.x);  // Phi_{k-1} - Phi_k exactly
    df dm1 = two_sum(zwall0 ? zsl * p_cur.y : pprev.y, -p_cur.y);
    const float* qp = PLO ? Plo + (size_t)k0 * sz + c0 : nullptr;
    float2 q_prev = make_float2(0.f, 0.f), q_cur = make_float2(0.f, 0.f);
    if (PLO) {
      q_prev = ld2(Plo + (size_t)kprev * sz + c0);
      q_cur = ld2(qp);
    }
    // ring of the next PF planes' f and Phi_{k+1} (loads issued PF planes ahead of their use)
    constexpr int PF = 2;
    double2 fr[PF];
    float2 pr[PF];
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      const int k = k0 + u;
      if (k < k1) {
        fr[u] = *reinterpret_cast<const double2*>(fp + (size_t)u * sz);
        pr[u] = (k == nz - 1) ? ld2(Phi + c0) : ld2(pp + (size_t)(u + 1) * sz);  // periodic wrap
      }
    }
    float nxm = pp[dxm], nxp = pp[dxp];
    float2 nym = ld2(pp + dym), nyp = ld2(pp + dyp);
    // r at one point from its six neighbours (Phi part, double-float); dm: Phi_{k-1} - Phi_k in,
    // Phi_k - Phi_{k+1} out
    auto point = [&](float xm, float xp, float ym, float yp, float pc, float zp, df& dm, const float4& co,
                     double fk) {
      const df dp = two_sum(zp, -pc);
      df L;
      if (S.iso) {
        const df sx = two_sum(xm, xp);
        const df sy = two_sum(ym, yp);
        const df s2 = two_sum(sx.hi, sy.hi);
        const df d = two_sum(s2.hi, -4.f * pc);
        L = df_prod(S.idx2, df_make(d.hi, __fadd_rn(d.lo, __fadd_rn(s2.lo, __fadd_rn(sx.lo, sy.lo)))));
      } else {
        L = df_prod(S.idx2, second_difference(xm, xp, pc));
        L = df_add_prod(L, S.idy2, second_difference(ym, yp, pc));
      }
      L = df_add_prod(L, df_make(co.x, co.y), dp);
      L = df_add_prod(L, df_make(co.z, co.w), dm);
      if (SHIFT) L = df_add_prod(L, S.shift, df_make(pc, 0.f));
      const df fs = df_split_rz(fk);
      dm = df_make(-dp.hi, -dp.lo);
      return __fadd_rn(__fsub_rn(fs.hi, L.hi), __fsub_rn(fs.lo, L.lo));
    };
    for (int kb = k0; kb < k1; kb += PF) {
#pragma unroll
      for (int u = 0; u < PF; ++u) {
        const int k = kb + u;
        if (k < k1) {
          const bool top = (k == nz - 1);
          const float2 p_next = pr[u];
          const double2 fk = fr[u];
          if (k + PF < k1) {
            fr[u] = *reinterpret_cast<const double2*>(fp + (size_t)PF * sz);
            pr[u] = (k + PF == nz - 1) ? ld2(Phi + c0) : ld2(pp + (size_t)(PF + 1) * sz);
          }
          const float xm0 = gxm ? sxm * p_cur.x : nxm;
          const float xp1 = gxp ? sxp * p_cur.y : nxp;
          const float ym0 = gym ? sym * p_cur.x : nym.x, ym1 = gym ? sym * p_cur.y : nym.y;
          const float yp0 = gyp ? syp * p_cur.x : nyp.x, yp1 = gyp ? syp * p_cur.y : nyp.y;
          if (k + 1 < k1) {
            nxm = pp[sz + dxm];
            nxp = pp[sz + dxp];
            nym = ld2(pp + sz + dym);
            nyp = ld2(pp + sz + dyp);
          }
          const bool ztop = BZ != BC_P && top;
          const float zp0 = ztop ? zsh * p_cur.x : p_next.x, zp1 = ztop ? zsh * p_cur.y : p_next.y;
          const float4 co = zc[k - k0];
          float r0 = point(xm0, p_cur.y, ym0, yp0, p_cur.x, zp0, dm0, co, fk.x);
          float r1 = point(p_cur.x, xp1, ym1, yp1, p_cur.y, zp1, dm1, co, fk.y);
          if (PLO) {
            const long long dzp = top ? -(long long)(nz - 1) * sz : (long long)sz;
            const float2 q_next = ld2(qp + dzp);
            const float qxm0 = gxm ? sxm * q_cur.x : qp[dxm];
            const float qxp1 = gxp ? sxp * q_cur.y : qp[dxp];
            const float2 qym = ld2(qp + dym), qyp = ld2(qp + dyp);
            const float qym0 = gym ? sym * q_cur.x : qym.x, qym1 = gym ? sym * q_cur.y : qym.y;
            const float qyp0 = gyp ? syp * q_cur.x : qyp.x, qyp1 = gyp ? syp * q_cur.y : qyp.y;
            const bool zbot = BZ != BC_P && k == 0;
            const float qzm0 = zbot ? zsl * q_cur.x : q_prev.x, qzm1 = zbot ? zsl * q_cur.y : q_prev.y;
            const float qzp0 = ztop ? zsh * q_cur.x : q_next.x, qzp1 = ztop ? zsh * q_cur.y : q_next.y;
            r0 -= S.idx2.hi * (qxm0 + q_cur.y - 2.f * q_cur.x) + S.idy2.hi * (qym0 + qyp0 - 2.f * q_cur.x) +
                  co.x * (qzp0 - q_cur.x) + co.z * (qzm0 - q_cur.x) + (SHIFT ? S.shift.hi * q_cur.x : 0.f);
            r1 -= S.idx2.hi * (q_cur.x + qxp1 - 2.f * q_cur.y) + S.idy2.hi * (qym1 + qyp1 - 2.f * q_cur.y) +
                  co.x * (qzp1 - q_cur.y) + co.z * (qzm1 - q_cur.y) + (SHIFT ? S.shift.hi * q_cur.y : 0.f);
            q_prev = q_cur;
            q_cur = q_next;
            qp += sz;
          }
          *reinterpret_cast<float2*>(rp) = make_float2(r0, r1);
          acc = __fmaf_rn(r0, r0, __fmaf_rn(r1, r1, acc));
          p_cur = p_next;
          pp += sz;
          fp += sz;
          rp += sz;
        }
      }
    }
  }
  if (norm_acc != nullptr) {
    __shared__ float red[R2X * R2Y / 32];
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
    const int t = threadIdx.y * R2X + threadIdx.x;
    if ((t & 31) == 0) red[t >> 5] = acc;
    __syncthreads();
    if (t == 0) {
      float s = 0.f;
      for (int w = 0; w < R2X * R2Y / 32; ++w) s += red[w];
      atomicAdd(norm_acc, (double)s);
    }
  }
}

// Four x-consecutive points per thread (nx a multiple of 4, f 16-byte and the float fields 16-byte
// aligned): Phi, Plo, r and the y neighbours move as float4, f as two double2; the address, loop and
// ghost work of a plane is shared by four points.  Same arithmetic per point as res_kernel.
constexpr int R4X = 32, R4Y = 8;  // threads of a CTA; a thread owns points i .. i + 3

template <int PM, int BX, int BY, int BZ>
__global__ void __launch_bounds__(R4X * R4Y, 2) res4_kernel(const double* __restrict__ f, const float* __restrict__ Phi,
                                                         const float* __restrict__ Plo, float* __restrict__ r,
                                                         StencilDF S, int kchunk, double* norm_acc) {
  constexpr bool PLO = (PM & 1) != 0, SHIFT = (PM & 2) != 0;
  __shared__ float4 zc[64];  // (c_k hi, c_k lo, a_k hi, a_k lo) of the chunk's planes
  const int nx = S.n[0], ny = S.n[1], nz = S.n[2];
  const int k0 = blockIdx.z * kchunk, k1 = min(nz, k0 + kchunk);
  for (int q = threadIdx.y * R4X + threadIdx.x; q < k1 - k0; q += R4X * R4Y)
    zc[q] = make_float4(S.sc_hi[k0 + q], S.sc_lo[k0 + q], S.sa_hi[k0 + q], S.sa_lo[k0 + q]);
  __syncthreads();
  const int i = 4 * (blockIdx.x * R4X + threadIdx.x), j = blockIdx.y * R4Y + threadIdx.y;
  float acc = 0.f;
  if (i < nx && j < ny) {  // nx is a multiple of 4, so i + 3 < nx as well
    const int sz = nx * ny;
    const int im = (i == 0) ? nx - 1 : i - 1, ip = (i + 4 == nx) ? 0 : i + 4;  // outer x neighbours
    const int jm = (j == 0) ? ny - 1 : j - 1, jp = (j == ny - 1) ? 0 : j + 1;
    const bool gxm = BX != BC_P && i == 0, gxp = BX != BC_P && i + 4 == nx;
    const bool gym = BY != BC_P && j == 0, gyp = BY != BC_P && j == ny - 1;
    const float sxm = (BX == BC_NN) ? 1.f : (BX == BC_DD) ? -1.f : ((S.xlo == BC_NN) ? 1.f : -1.f);
    const float sxp = (BX == BC_NN) ? 1.f : (BX == BC_DD) ? -1.f : ((S.xhi == BC_NN) ? 1.f : -1.f);
    const float sym = (BY == BC_NN) ? 1.f : (BY == BC_DD) ? -1.f : ((S.ylo == BC_NN) ? 1.f : -1.f);
    const float syp = (BY == BC_NN) ? 1.f : (BY == BC_DD) ? -1.f : ((S.yhi == BC_NN) ? 1.f : -1.f);
    const float zsl = (BZ == BC_NN) ? 1.f : (BZ == BC_DD) ? -1.f : ((S.zlo == BC_NN) ? 1.f : -1.f);
    const float zsh = (BZ == BC_NN) ? 1.f : (BZ == BC_DD) ? -1.f : ((S.zhi == BC_NN) ? 1.f : -1.f);
    const int c0 = j * nx + i;
    const int dxm = im - i, dxp = ip - i, dym = (jm - j) * nx, dyp = (jp - j) * nx;
    const int kprev = (k0 == 0) ? nz - 1 : k0 - 1;
    const float* pp = Phi + (size_t)k0 * sz + c0;
    const double* fp = f + (size_t)k0 * sz + c0;
    float* rp = r + (size_t)k0 * sz + c0;
    auto ld4 = [](const float* a) { return *reinterpret_cast<const float4*>(a); };
    float4 p_cur = ld4(pp);
    const bool zwall0 = BZ != BC_P && k0 == 0;
    df dm[4];
    {
      const float4 pv = ld4(Phi + (size_t)kprev * sz + c0);
      const float pvs[4] = {pv.x, pv.y, pv.z, pv.w}, pcs[4] = {p_cur.x, p_cur.y, p_cur.z, p_cur.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) dm[e] = two_sum(zwall0 ? zsl * pcs[e] : pvs[e], -pcs[e]);  // Phi_{k-1} - Phi_k
    }
    const float* qp = PLO ? Plo + (size_t)k0 * sz + c0 : nullptr;
    float4 q_prev = make_float4(0.f, 0.f, 0.f, 0.f), q_cur = q_prev;
    if (PLO) {
      q_prev = ld4(Plo + (size_t)kprev * sz + c0);
      q_cur = ld4(qp);
    }
    // ring of the next PF planes' f and Phi_{k+1} (loads issued PF planes ahead of their use)
    constexpr int PF = 2;
    double2 fa[PF], fb[PF];
    float4 pr[PF];
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      const int k = k0 + u;
      if (k < k1) {
        fa[u] = *reinterpret_cast<const double2*>(fp + (size_t)u * sz);
        fb[u] = *reinterpret_cast<const double2*>(fp + (size_t)u * sz + 2);
        pr[u] = (k == nz - 1) ? ld4(Phi + c0) : ld4(pp + (size_t)(u + 1) * sz);  // periodic wrap
      }
    }
    float nxm = pp[dxm], nxp = pp[dxp];
    float4 nym = ld4(pp + dym), nyp = ld4(pp + dyp);
    // r at one point from its six neighbours (Phi part, double-float); dm: Phi_{k-1} - Phi_k in,
    // Phi_k - Phi_{k+1} out
    auto point = [&](float xm, float xp, float ym, float yp, float pc, float zp, df& dmv, const float4& co,
                     double fk) {
      const df dp = two_sum(zp, -pc);
      df L;
      if (S.iso) {
        const df sx = two_sum(xm, xp);
        const df sy = two_sum(ym, yp);
        const df s2 = two_sum(sx.hi, sy.hi);
        const df d = two_sum(s2.hi, -4.f * pc);
        L = df_prod(S.idx2, df_make(d.hi, __fadd_rn(d.lo, __fadd_rn(s2.lo, __fadd_rn(sx.lo, sy.lo)))));
      } else {
        L = df_prod(S.idx2, second_difference(xm, xp, pc));
        L = df_add_prod(L, S.idy2, second_difference(ym, yp, pc));
      }
      L = df_add_prod(L, df_make(co.x, co.y), dp);
      L = df_add_prod(L, df_make(co.z, co.w), dmv);
      if (SHIFT) L = df_add_prod(L, S.shift, df_make(pc, 0.f));
      const df fs = df_split_rz(fk);
      dmv = df_make(-dp.hi, -dp.lo);
      return __fadd_rn(__fsub_rn(fs.hi, L.hi), __fsub_rn(fs.lo, L.lo));
    };
    for (int kb = k0; kb < k1; kb += PF) {
#pragma unroll
      for (int u = 0; u < PF; ++u) {
        const int k = kb + u;
        if (k < k1) {
          const bool top = (k == nz - 1);
          const float4 p_next = pr[u];
          const double2 f01 = fa[u], f23 = fb[u];
          if (k + PF < k1) {
            fa[u] = *reinterpret_cast<const double2*>(fp + (size_t)PF * sz);
            fb[u] = *reinterpret_cast<const double2*>(fp + (size_t)PF * sz + 2);
            pr[u] = (k + PF == nz - 1) ? ld4(Phi + c0) : ld4(pp + (size_t)(PF + 1) * sz);
          }
          const float pcs[4] = {p_cur.x, p_cur.y, p_cur.z, p_cur.w};
          const float yms[4] = {nym.x, nym.y, nym.z, nym.w}, yps[4] = {nyp.x, nyp.y, nyp.z, nyp.w};
          const float zps[4] = {p_next.x, p_next.y, p_next.z, p_next.w};
          const float xl = gxm ? sxm * p_cur.x : nxm;
          const float xr = gxp ? sxp * p_cur.w : nxp;
          if (k + 1 < k1) {
            nxm = pp[sz + dxm];
            nxp = pp[sz + dxp];
            nym = ld4(pp + sz + dym);
            nyp = ld4(pp + sz + dyp);
          }
          const bool ztop = BZ != BC_P && top;
          const float4 co = zc[k - k0];
          const double fks[4] = {f01.x, f01.y, f23.x, f23.y};
          float rr[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float c = pcs[e];
            const float xm = (e == 0) ? xl : pcs[(e + 3) & 3];
            const float xp = (e == 3) ? xr : pcs[(e + 1) & 3];
            const float ym = gym ? sym * c : yms[e];
            const float yp = gyp ? syp * c : yps[e];
            const float zp = ztop ? zsh * c : zps[e];
            rr[e] = point(xm, xp, ym, yp, c, zp, dm[e], co, fks[e]);
          }
          if (PLO) {
            const long long dzp = top ? -(long long)(nz - 1) * sz : (long long)sz;
            const float4 q_next = ld4(qp + dzp);
            const float4 qym4 = ld4(qp + dym), qyp4 = ld4(qp + dyp);
            const float qcs[4] = {q_cur.x, q_cur.y, q_cur.z, q_cur.w};
            const float qyms[4] = {qym4.x, qym4.y, qym4.z, qym4.w}, qyps[4] = {qyp4.x, qyp4.y, qyp4.z, qyp4.w};
            const float qzms[4] = {q_prev.x, q_prev.y, q_prev.z, q_prev.w};
            const float qzps[4] = {q_next.x, q_next.y, q_next.z, q_next.w};
            const float qxl = gxm ? sxm * q_cur.x : qp[dxm];
            const float qxr = gxp ? sxp * q_cur.w : qp[dxp];
            const bool zbot = BZ != BC_P && k == 0;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float c = qcs[e];
              const float qxm = (e == 0) ? qxl : qcs[(e + 3) & 3];
              const float qxp = (e == 3) ? qxr : qcs[(e + 1) & 3];
              const float qym = gym ? sym * c : qyms[e];
              const float qyp = gyp ? syp * c : qyps[e];
              const float qzm = zbot ? zsl * c : qzms[e];
              const float qzp = ztop ? zsh * c : qzps[e];
              rr[e] -= S.idx2.hi * (qxm + qxp - 2.f * c) + S.idy2.hi * (qym + qyp - 2.f * c) + co.x * (qzp - c) +
                       co.z * (qzm - c) + (SHIFT ? S.shift.hi * c : 0.f);
            }
            q_prev = q_cur;
            q_cur = q_next;
            qp += sz;
          }
          *reinterpret_cast<float4*>(rp) = make_float4(rr[0], rr[1], rr[2], rr[3]);
          acc = __fmaf_rn(rr[0], rr[0], __fmaf_rn(rr[1], rr[1], __fmaf_rn(rr[2], rr[2], __fmaf_rn(rr[3], rr[3], acc))));
          p_cur = p_next;
          pp += sz;
          fp += sz;
          rp += sz;
        }
      }
    }
  }
  if (norm_acc != nullptr) {
    __shared__ float red[R4X * R4Y / 32];
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
    const int t = threadIdx.y * R4X + threadIdx.x;
    if ((t & 31) == 0) red[t >> 5] = acc;
    __syncthreads();
    if (t == 0) {
      float s = 0.f;
      for (int w = 0; w < R4X * R4Y / 32; ++w) s += red[w];
      atomicAdd(norm_acc, (double)s);
    }
  }
}

template <int PLO, int BX, int BY, int BZ>
cudaError_t res_launch(dim3 grid, dim3 block, const double* f, const float* Phi, const float* Plo, float* r,
                       const StencilDF& S, int kchunk, double* acc, cudaStream_t st, int pts) {
  if (pts == 4)
    res4_kernel<PLO, BX, BY, BZ><<<grid, block, 0, st>>>(f, Phi, Plo, r, S, kchunk, acc);
  else if (pts == 2)
    res2_kernel<PLO, BX, BY, BZ><<<grid, block, 0, st>>>(f, Phi, Plo, r, S, kchunk, acc);
  else
    res_kernel<PLO, BX, BY, BZ><<<grid, block, 0, st>>>(f, Phi, Plo, r, S, kchunk, acc);
  return cudaGetLastError();
}

template <int PLO, int BX, int BY>
cudaError_t res_bz(int bz, dim3 g, dim3 b, const double* f, const float* Phi, const float* Plo, float* r,
                   const StencilDF& S, int kc, double* acc, cudaStream_t st, int pr) {
  if (bz == BC_P) return res_launch<PLO, BX, BY, BC_P>(g, b, f, Phi, Plo, r, S, kc, acc, st, pr);
  if (bz == BC_NN) return res_launch<PLO, BX, BY, BC_NN>(g, b, f, Phi, Plo, r, S, kc, acc, st, pr);
  if (bz == BC_DD) return res_launch<PLO, BX, BY, BC_DD>(g, b, f, Phi, Plo, r, S, kc, acc, st, pr);
  return res_launch<PLO, BX, BY, BC_ND>(g, b, f, Phi, Plo, r, S, kc, acc, st, pr);  // either mixed pair
}
template <int PLO, int BX>
cudaError_t res_by(int by, int bz, dim3 g, dim3 b, const double* f, const float* Phi, const float* Plo, float* r,
                   const StencilDF& S, int kc, double* acc, cudaStream_t st, int pr) {
  if (by == BC_P) return res_bz<PLO, BX, BC_P>(bz, g, b, f, Phi, Plo, r, S, kc, acc, st, pr);
  if (by == BC_NN) return res_bz<PLO, BX, BC_NN>(bz, g, b, f, Phi, Plo, r, S, kc, acc, st, pr);
  if (by == BC_DD) return res_bz<PLO, BX, BC_DD>(bz, g, b, f, Phi, Plo, r, S, kc, acc, st, pr);
  return res_bz<PLO, BX, BC_ND>(bz, g, b, f, Phi, Plo, r, S, kc, acc, st, pr);  // either mixed pair
}
template <int PLO>
cudaError_t res_bx(const int* bc, dim3 g, dim3 b, const double* f, const float* Phi, const float* Plo, float* r,
                   const StencilDF& S, int kc, double* acc, cudaStream_t st, int pr) {
  if (bc[0] == BC_P) return res_by<PLO, BC_P>(bc[1], bc[2], g, b, f, Phi, Plo, r, S, kc, acc, st, pr);
  if (bc[0] == BC_NN) return res_by<PLO, BC_NN>(bc[1], bc[2], g, b, f, Phi, Plo, r, S, kc, acc, st, pr);
  if (bc[0] == BC_DD) return res_by<PLO, BC_DD>(bc[1], bc[2], g, b, f, Phi, Plo, r, S, kc, acc, st, pr);
  return res_by<PLO, BC_ND>(bc[1], bc[2], g, b, f, Phi, Plo, r, S, kc, acc, st, pr);
}

}  // namespace

cudaError_t launch_residual(const cans_plan_s* P, const double* f, const float* Phi, const float* Plo, bool plo,
                            float* r, double* norm_acc, cudaStream_t st) {
  const int nx = P->n[0], ny = P->n[1], nz = P->n[2];
  const int kchunk = std::min(nz, 64);  // at most the 64 planes whose z coefficients a CTA stages
  dim3 grid((nx + RX - 1) / RX, (ny + RY - 1) / RY, (nz + kchunk - 1) / kchunk);
  dim3 block(RX, RY);
  // four (or two) points per thread where nx allows and the vector accesses are aligned
  const uintptr_t fl = reinterpret_cast<uintptr_t>(Phi) | reinterpret_cast<uintptr_t>(r) |
                       (plo ? reinterpret_cast<uintptr_t>(Plo) : 0);
  const bool f16 = (reinterpret_cast<uintptr_t>(f) & 15) == 0;
  int pts = 1;
  if (P->res_pts >= 4 && nx % 4 == 0 && f16 && (fl & 15) == 0)
    pts = 4;
  else if (P->res_pts >= 2 && nx % 2 == 0 && f16 && (fl & 7) == 0)
    pts = 2;
  if (pts == 4) {
    grid.x = (nx / 4 + R4X - 1) / R4X;
    block = dim3(R4X, R4Y);
  } else if (pts == 2) {
    grid.x = (nx / 2 + R2X - 1) / R2X;
    block = dim3(R2X, R2Y);
  }
  const StencilDF S = stencil_df(P);
  const int pm = (plo ? 1 : 0) | (S.shift.hi != 0.f ? 2 : 0);
  switch (pm) {
    case 0: return res_bx<0>(P->bc, grid, block, f, Phi, Plo, r, S, kchunk, norm_acc, st, pts);
    case 1: return res_bx<1>(P->bc, grid, block, f, Phi, Plo, r, S, kchunk, norm_acc, st, pts);
    case 2: return res_bx<2>(P->bc, grid, block, f, Phi, Plo, r, S, kchunk, norm_acc, st, pts);
    default: return res_bx<3>(P->bc, grid, block, f, Phi, Plo, r, S, kchunk, norm_acc, st, pts);
  }
}

}  // namespace cans
