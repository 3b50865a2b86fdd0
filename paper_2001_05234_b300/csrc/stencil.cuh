// The 7-point operator of Eq. poi (plus the Helmholtz shift of Eq. up_id_2, when set) applied to
// the mixed path's iterate Phi + Plo (two float fields) and subtracted from f (double): the residual of a refinement sweep, evaluated in
// double-float arithmetic so that it carries about 47 significant bits although every operand is
// read as a float (f is split on the fly).
#pragma once
#include <cuda_runtime.h>

#include "dfloat.cuh"
#include "plan.cuh"

namespace cans {

// acc - coef * x for double-float acc, coef and x: the product's error-free head and a float tail.
__device__ __forceinline__ df df_sub_prod(df acc, df coef, df x) {
  df p = two_prod(coef.hi, x.hi);
  p.lo = __fmaf_rn(coef.hi, x.lo, __fmaf_rn(coef.lo, x.hi, p.lo));
  const df s = two_sum(acc.hi, -p.hi);
  return df_make(s.hi, __fadd_rn(s.lo, __fsub_rn(acc.lo, p.lo)));
}

// xm + xp - 2 c as an (almost exact) double-float: two error-free sums
__device__ __forceinline__ df second_difference(float xm, float xp, float c) {
  const df a = two_sum(xm, xp);
  const df b = two_sum(a.hi, -2.f * c);
  return df_make(b.hi, __fadd_rn(b.lo, a.lo));
}

// Wall ghost of a cell-centred value: Neumann mirrors it, Dirichlet mirrors it with the sign flipped.
__device__ __forceinline__ float wall_ghost(int bc, float c) { return (bc == BC_NN) ? c : -c; }

// r = f - L_h(Phi + Plo) at cell (i, j, k) (Eq. poi): the Phi part in double-float arithmetic, the
// small Plo part in float (skipped when PLO is false, i.e. Plo is known to be zero).
template <bool PLO>
__device__ __forceinline__ float residual_point(const double* __restrict__ f, const float* __restrict__ Phi,
                                                const float* __restrict__ Plo, const StencilDF& S, size_t c, int i,
                                                int j, int k) {
  const int nx = S.n[0], ny = S.n[1], nz = S.n[2];
  const long long sz = (long long)nx * ny;
  // neighbour offsets with periodic wrap; at a wall the loaded value is replaced by the ghost
  const int oxm = (i == 0) ? nx - 1 : -1, oxp = (i == nx - 1) ? 1 - nx : 1;
  const int oym = (j == 0) ? (ny - 1) * nx : -nx, oyp = (j == ny - 1) ? (1 - ny) * nx : nx;
  const long long ozm = (k == 0) ? (nz - 1) * sz : -sz, ozp = (k == nz - 1) ? (1 - nz) * sz : sz;
  const float* q = Phi + c;
  const float pc = q[0];
  float xm = q[oxm], xp = q[oxp], ym = q[oym], yp = q[oyp], zm = q[ozm], zp = q[ozp];
  if (S.bc[0] != BC_P) {
    if (i == 0) xm = wall_ghost(S.xlo, pc);
    if (i == nx - 1) xp = wall_ghost(S.xhi, pc);
  }
  if (S.bc[1] != BC_P) {
    if (j == 0) ym = wall_ghost(S.ylo, pc);
    if (j == ny - 1) yp = wall_ghost(S.yhi, pc);
  }
  if (S.bc[2] != BC_P) {
    if (k == 0) zm = wall_ghost(S.zlo, pc);
    if (k == nz - 1) zp = wall_ghost(S.zhi, pc);
  }
  df acc = df_from_double(f[c]);
  acc = df_sub_prod(acc, S.idx2, second_difference(xm, xp, pc));
  acc = df_sub_prod(acc, S.idy2, second_difference(ym, yp, pc));
  acc = df_sub_prod(acc, df_make(S.sc_hi[k], S.sc_lo[k]), two_sum(zp, -pc));
  acc = df_sub_prod(acc, df_make(S.sa_hi[k], S.sa_lo[k]), two_sum(zm, -pc));
  if (S.shift.hi != 0.f) acc = df_sub_prod(acc, S.shift, df_make(pc, 0.f));
  float r = acc.hi + acc.lo;
  if (PLO) {
    const float* o = Plo + c;
    const float qc = o[0];
    float qxm = o[oxm], qxp = o[oxp], qym = o[oym], qyp = o[oyp], qzm = o[ozm], qzp = o[ozp];
    if (S.bc[0] != BC_P) {
      if (i == 0) qxm = wall_ghost(S.xlo, qc);
      if (i == nx - 1) qxp = wall_ghost(S.xhi, qc);
    }
    if (S.bc[1] != BC_P) {
      if (j == 0) qym = wall_ghost(S.ylo, qc);
      if (j == ny - 1) qyp = wall_ghost(S.yhi, qc);
    }
    if (S.bc[2] != BC_P) {
      if (k == 0) qzm = wall_ghost(S.zlo, qc);
      if (k == nz - 1) qzp = wall_ghost(S.zhi, qc);
    }
    r -= S.idx2.hi * (qxm + qxp - 2.f * qc) + S.idy2.hi * (qym + qyp - 2.f * qc) + S.sc_hi[k] * (qzp - qc) +
         S.sa_hi[k] * (qzm - qc) + S.shift.hi * qc;
  }
  return r;
}

// The residual at the two cells (i, j, k), (i+1, j, k) of one packed x-pair (i even): the y and z
// neighbours come as float2 loads, the wrap/ghost logic is evaluated once, f as one double2 load.
// When 1/dx^2 == 1/dy^2 (S.iso) the x and y second differences are summed exactly first and
// multiplied once.  Same arithmetic otherwise as residual_point.
__device__ __forceinline__ float2 ld_f2(const float* p) { return *reinterpret_cast<const float2*>(p); }

template <bool PLO>
__device__ __forceinline__ float2 residual_pair(const double* __restrict__ f, const float* __restrict__ Phi,
                                                const float* __restrict__ Plo, const StencilDF& S, size_t c, int i,
                                                int j, int k) {
  const int nx = S.n[0], ny = S.n[1], nz = S.n[2];
  const long long sz = (long long)nx * ny;
  const int oym = (j == 0) ? (ny - 1) * nx : -nx, oyp = (j == ny - 1) ? (1 - ny) * nx : nx;
  const long long ozm = (k == 0) ? (nz - 1) * sz : -sz, ozp = (k == nz - 1) ? (1 - nz) * sz : sz;
  const int oxm = (i == 0) ? nx - 1 : -1, oxp = (i + 1 == nx - 1) ? 2 - nx : 2;  // left of i, right of i+1
  const bool wx = S.bc[0] != BC_P, wy = S.bc[1] != BC_P, wz = S.bc[2] != BC_P;
  const double2 fd = *reinterpret_cast<const double2*>(f + c);
  const float sca = S.sc_hi[k], scl = S.sc_lo[k], saa = S.sa_hi[k], sal = S.sa_lo[k];
  float r[2];
  {
    const float* q = Phi + c;
    const float2 pc = ld_f2(q), ym2 = ld_f2(q + oym), yp2 = ld_f2(q + oyp), zm2 = ld_f2(q + ozm), zp2 = ld_f2(q + ozp);
    float xl = q[oxm], xr = q[oxp];
    if (wx && i == 0) xl = wall_ghost(S.xlo, pc.x);
    if (wx && i + 1 == nx - 1) xr = wall_ghost(S.xhi, pc.y);
    const float pcs[2] = {pc.x, pc.y}, xms[2] = {xl, pc.x}, xps[2] = {pc.y, xr};
    const float yms[2] = {ym2.x, ym2.y}, yps[2] = {yp2.x, yp2.y}, zms[2] = {zm2.x, zm2.y}, zps[2] = {zp2.x, zp2.y};
    const double fs[2] = {fd.x, fd.y};
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const float c0 = pcs[e];
      const float ym = (wy && j == 0) ? wall_ghost(S.ylo, c0) : yms[e];
      const float yp = (wy && j == ny - 1) ? wall_ghost(S.yhi, c0) : yps[e];
      const float zm = (wz && k == 0) ? wall_ghost(S.zlo, c0) : zms[e];
      const float zp = (wz && k == nz - 1) ? wall_ghost(S.zhi, c0) : zps[e];
      df acc = df_split(fs[e]);
      if (S.iso) {
        const df a = two_sum(xms[e], xps[e]);
        const df b = two_sum(ym, yp);
        const df s2 = two_sum(a.hi, b.hi);
        const df d = two_sum(s2.hi, -4.f * c0);
        acc = df_sub_prod(acc, S.idx2, df_make(d.hi, __fadd_rn(d.lo, __fadd_rn(s2.lo, __fadd_rn(a.lo, b.lo)))));
      } else {
        acc = df_sub_prod(acc, S.idx2, second_difference(xms[e], xps[e], c0));
        acc = df_sub_prod(acc, S.idy2, second_difference(ym, yp, c0));
      }
      acc = df_sub_prod(acc, df_make(sca, scl), two_sum(zp, -c0));
      acc = df_sub_prod(acc, df_make(saa, sal), two_sum(zm, -c0));
      if (S.shift.hi != 0.f) acc = df_sub_prod(acc, S.shift, df_make(c0, 0.f));
      r[e] = acc.hi + acc.lo;
    }
  }
  if (PLO) {
    const float* o = Plo + c;
    const float2 qc = ld_f2(o), ym2 = ld_f2(o + oym), yp2 = ld_f2(o + oyp), zm2 = ld_f2(o + ozm), zp2 = ld_f2(o + ozp);
    float xl = o[oxm], xr = o[oxp];
    if (wx && i == 0) xl = wall_ghost(S.xlo, qc.x);
    if (wx && i + 1 == nx - 1) xr = wall_ghost(S.xhi, qc.y);
    const float qcs[2] = {qc.x, qc.y}, xms[2] = {xl, qc.x}, xps[2] = {qc.y, xr};
    const float yms[2] = {ym2.x, ym2.y}, yps[2] = {yp2.x, yp2.y}, zms[2] = {zm2.x, zm2.y}, zps[2] = {zp2.x, zp2.y};
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const float c0 = qcs[e];
      const float ym = (wy && j == 0) ? wall_ghost(S.ylo, c0) : yms[e];
      const float yp = (wy && j == ny - 1) ? wall_ghost(S.yhi, c0) : yps[e];
      const float zm = (wz && k == 0) ? wall_ghost(S.zlo, c0) : zms[e];
      const float zp = (wz && k == nz - 1) ? wall_ghost(S.zhi, c0) : zps[e];
      r[e] -= S.idx2.hi * (xms[e] + xps[e] - 2.f * c0) + S.idy2.hi * (ym + yp - 2.f * c0) + sca * (zp - c0) +
              saa * (zm - c0) + S.shift.hi * c0;
    }
  }
  return make_float2(r[0], r[1]);
}

}  // namespace cans
