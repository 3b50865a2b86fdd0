// The 7-point operator of Eq. poi applied to the mixed path's iterate Phi + Plo (two float
// fields) and subtracted from f (double): the residual of a refinement sweep, evaluated in
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
    if (i == 0) xm = wall_ghost(S.bc[0], pc);
    if (i == nx - 1) xp = wall_ghost(S.bc[0], pc);
  }
  if (S.bc[1] != BC_P) {
    if (j == 0) ym = wall_ghost(S.bc[1], pc);
    if (j == ny - 1) yp = wall_ghost(S.bc[1], pc);
  }
  if (S.bc[2] != BC_P) {
    if (k == 0) zm = wall_ghost(S.bc[2], pc);
    if (k == nz - 1) zp = wall_ghost(S.bc[2], pc);
  }
  df acc = df_from_double(f[c]);
  acc = df_sub_prod(acc, S.idx2, second_difference(xm, xp, pc));
  acc = df_sub_prod(acc, S.idy2, second_difference(ym, yp, pc));
  acc = df_sub_prod(acc, df_make(S.sc_hi[k], S.sc_lo[k]), two_sum(zp, -pc));
  acc = df_sub_prod(acc, df_make(S.sa_hi[k], S.sa_lo[k]), two_sum(zm, -pc));
  float r = acc.hi + acc.lo;
  if (PLO) {
    const float* o = Plo + c;
    const float qc = o[0];
    float qxm = o[oxm], qxp = o[oxp], qym = o[oym], qyp = o[oyp], qzm = o[ozm], qzp = o[ozp];
    if (S.bc[0] != BC_P) {
      if (i == 0) qxm = wall_ghost(S.bc[0], qc);
      if (i == nx - 1) qxp = wall_ghost(S.bc[0], qc);
    }
    if (S.bc[1] != BC_P) {
      if (j == 0) qym = wall_ghost(S.bc[1], qc);
      if (j == ny - 1) qyp = wall_ghost(S.bc[1], qc);
    }
    if (S.bc[2] != BC_P) {
      if (k == 0) qzm = wall_ghost(S.bc[2], qc);
      if (k == nz - 1) qzp = wall_ghost(S.bc[2], qc);
    }
    r -= S.idx2.hi * (qxm + qxp - 2.f * qc) + S.idy2.hi * (qym + qyp - 2.f * qc) + S.sc_hi[k] * (qzp - qc) +
         S.sa_hi[k] * (qzm - qc);
  }
  return r;
}

}  // namespace cans
