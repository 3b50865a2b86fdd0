// Fractional-step kernels around the Poisson solve (Numerical method: Eq. up, Eq. poi_ns, the
// correction u = u* - gamma dt G Phi and the pressure update p += Phi; Eq. dt and its chkdt
// listing; constant-flow-rate forcing of the Validation section), for a channel: x and y periodic,
// no-slip walls at z = 0 and z = Lz.
//
// Staggered arrays, Nx x Ny x Nz, x fastest: u on the x-face between cells i and i+1, v on the y-face
// between j and j+1, w on the z-face between k and k+1 (w[Nz-1] is the top wall and stays 0), p at
// cell centres.  Advection: conservative divergence of u (x) u with two-point averages; diffusion:
// 3-point Laplacian with no-slip ghosts (ghost = -interior).  Everything in FP64.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "plan.cuh"

namespace cans {

struct Chan {
  int nx, ny, nz;
  double dxi, dyi;            // 1/dx, 1/dy
  const double* dzf;          // cell widths
  const double* dzfi;         // 1/dzf
  const double* dzci;         // 1/dzc_{k+1/2} (distance centre k to centre k+1; top: the wall ghost)
  __device__ __forceinline__ size_t id(int i, int j, int k) const {
    i = (i < 0) ? i + nx : (i >= nx ? i - nx : i);
    j = (j < 0) ? j + ny : (j >= ny ? j - ny : j);
    return (size_t)i + (size_t)nx * ((size_t)j + (size_t)ny * k);
  }
};

// tangential velocity with no-slip ghosts
__device__ __forceinline__ double Ut(const Chan& g, const double* a, int i, int j, int k) {
  if (k < 0) return -a[g.id(i, j, 0)];
  if (k >= g.nz) return -a[g.id(i, j, g.nz - 1)];
  return a[g.id(i, j, k)];
}
// wall-normal velocity (zero on both walls)
__device__ __forceinline__ double Wn(const Chan& g, const double* w, int i, int j, int k) {
  if (k < 0 || k >= g.nz - 1) return 0.0;
  return w[g.id(i, j, k)];
}
__device__ __forceinline__ double dzc_inv_below(const Chan& g, int k) {  // 1/dzc_{k-1/2}
  return (k == 0) ? g.dzfi[0] : g.dzci[k - 1];
}

__device__ __forceinline__ double lap_t(const Chan& g, const double* a, int i, int j, int k) {
  const double c = a[g.id(i, j, k)];
  const double lx = (a[g.id(i - 1, j, k)] - 2 * c + a[g.id(i + 1, j, k)]) * g.dxi * g.dxi;
  const double ly = (a[g.id(i, j - 1, k)] - 2 * c + a[g.id(i, j + 1, k)]) * g.dyi * g.dyi;
  const double lz =
      ((Ut(g, a, i, j, k + 1) - c) * g.dzci[k] - (c - Ut(g, a, i, j, k - 1)) * dzc_inv_below(g, k)) * g.dzfi[k];
  return lx + ly + lz;
}

// Momentum right-hand side A(u) + nu L(u) (Eq. up) and the predictor
//   u* = u + dt (alpha rhs + beta rhs_prev - gamma G p);  rhs replaces rhs_prev in place.
// IMPL (Crank-Nicolson diffusion, Eq. up_id and Eq. up_id_2): rhs = A(u) alone, and us receives the
// right-hand side of the Helmholtz problem (L + sigma) u* = sigma (u** - gamma nu dt/2 L u), sigma =
// -2/(gamma nu dt), which is sigma (u + dt (alpha A + beta A_prev - gamma G p)) - L u.
// Flux form, on tiles of MX x MY columns that march along z (a thread owns one (i, j) column and MZ
// planes of it).  The conservative advection of Eq. up is a difference of
// face and edge fluxes, and each flux serves the two points on either side of it -- and the uv, uw,
// vw edge fluxes two equations each -- so every flux is computed once:
//   A(i)  = (u_{i-1} + u_i)^2 at cell centres (x flux of u),  B(j) = (v_{j-1} + v_j)^2 (y flux of v),
//   C(k)  = (w_{k-1} + w_k)^2 (z flux of w),
//   Euv   = (u_j + u_{j+1})(v_i + v_{i+1}) on the x-y edges, Euw = (u_k + u_{k+1})(w_i + w_{i+1}) on the
//   x-z edges, Evw = (v_k + v_{k+1})(w_j + w_{j+1}) on the y-z edges,
// each thread forming those on its east, north and top sides.  The west and south ones come from the
// neighbouring threads through a shared tile (double-buffered by plane; the tile's first row and
// column form theirs themselves), the bottom ones from the thread's own previous plane, as do the z
// first differences of the diffusion.  Advection is the conservative central form with two-point
// averages (the 1/4 of the averages in the metric factors), diffusion the 3-point Laplacian with the
// no-slip ghosts -u for u and v and w = 0 on the walls.  B300 issues FP64 at 1/64 of the FP32 rate and
// the kernel is bound by it, so the shared fluxes, nu and dt folded into the coefficients, and one
// fused chain for nu L u - A(u) keep it at ~79 FP64 instructions per point (a pointwise form of the
// same operator took ~96 and 5.58 ms per 512 x 256 x 192 launch against 4.91).
constexpr int MX = 32, MY = 8, MZ = 16;

template <bool IMPL>
__global__ void __launch_bounds__(MX * MY, 2) momentum_flux_kernel(
    Chan g, const double* __restrict__ u, const double* __restrict__ v, const double* __restrict__ w,
    const double* __restrict__ p, double* __restrict__ ru, double* __restrict__ rv, double* __restrict__ rw,
    double* __restrict__ us, double* __restrict__ vs, double* __restrict__ ws, double nu, double alpha, double beta,
    double gamma, const double* __restrict__ dt_dev, double sigma) {
  // shared fluxes of the current plane, two buffers by plane parity: [A, Euv, Euw] read by the east
  // neighbour, [Euv, B, Evw] by the north one (Euv by both)
  __shared__ double sA[2][MY][MX], sUV[2][MY][MX], sUW[2][MY][MX], sB[2][MY][MX], sVW[2][MY][MX];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.x * MX + tx, j = blockIdx.y * MY + ty;
  const bool live = i < g.nx && j < g.ny;
  const int k0 = blockIdx.z * MZ, k1 = min(g.nz, k0 + MZ);
  const double dt = *dt_dev;
  const double qdx = 0.25 * g.dxi, qdy = 0.25 * g.dyi, dx2 = g.dxi * g.dxi, dy2 = g.dyi * g.dyi;
  const double ndx2 = nu * dx2, ndy2 = nu * dy2;
  const double dta = dt * alpha, dtb = dt * beta, dtg = -dt * gamma, dga_x = dtg * g.dxi, dga_y = dtg * g.dyi;
  const int ie = (i + 1 < g.nx) ? i + 1 : 0, iw = (i > 0) ? i - 1 : g.nx - 1;
  const int jn = (j + 1 < g.ny) ? j + 1 : 0, js = (j > 0) ? j - 1 : g.ny - 1;
  const size_t plane = (size_t)g.nx * g.ny;
  auto at = [&](int ii, int jj, int kk) { return (size_t)ii + (size_t)g.nx * ((size_t)jj + (size_t)g.ny * kk); };
  auto U = [&](const double* a, int ii, int jj, int kk) {  // tangential component with no-slip ghosts
    if (kk < 0) return -a[at(ii, jj, 0)];
    if (kk >= g.nz) return -a[at(ii, jj, g.nz - 1)];
    return a[at(ii, jj, kk)];
  };
  auto Wv = [&](int ii, int jj, int kk) { return (kk < 0 || kk >= g.nz - 1) ? 0.0 : w[at(ii, jj, kk)]; };
  // the carried bottom quantities of plane k (from plane k - 1): the z fluxes Euw, Evw and C at the
  // bottom face, and the bottom z first differences of u, v (scaled by 1/dzc) and w (by 1/dzf)
  double fuw_b = 0, fvw_b = 0, c_b = 0, gu_b = 0, gv_b = 0, hw_b = 0;
  if (live) {
    const int kb = k0 - 1;
    fuw_b = (U(u, i, j, kb) + U(u, i, j, k0)) * (Wv(i, j, kb) + Wv(ie, j, kb));
    fvw_b = (U(v, i, j, kb) + U(v, i, j, k0)) * (Wv(i, j, kb) + Wv(i, jn, kb));
    const double wb0 = Wv(i, j, kb), wb1 = Wv(i, j, k0);  // C at cell k0: (w_{k0-1} + w_{k0})^2
    c_b = (wb0 + wb1) * (wb0 + wb1);
    const double dzb = (k0 == 0) ? g.dzfi[0] : g.dzci[k0 - 1];
    gu_b = (U(u, i, j, k0) - U(u, i, j, kb)) * dzb;
    gv_b = (U(v, i, j, k0) - U(v, i, j, kb)) * dzb;
    hw_b = (wb1 - wb0) * g.dzfi[k0];  // w = 0 on the bottom wall face
  }
  for (int k = k0; k < k1; ++k) {
    const int b = k & 1;
    double uc = 0, vc = 0, wc = 0, ue = 0, un = 0, ut = 0, vE = 0, vn = 0, vt = 0, wE = 0, wn = 0, wt = 0;
    double fA_e = 0, fuv = 0, fuw = 0, fB_n = 0, fvw = 0, c_t = 0;
    const size_t c = at(i, j, k);
    if (live) {
      uc = u[c];
      vc = v[c];
      wc = Wv(i, j, k);
      ue = u[at(ie, j, k)];
      un = u[at(i, jn, k)];
      ut = U(u, i, j, k + 1);
      vE = v[at(ie, j, k)];
      vn = v[at(i, jn, k)];
      vt = U(v, i, j, k + 1);
      wE = Wv(ie, j, k);
      wn = Wv(i, jn, k);
      wt = Wv(i, j, k + 1);
      // this thread's east, north and top fluxes
      fA_e = (uc + ue) * (uc + ue);
      fuv = (uc + un) * (vc + vE);
      fuw = (uc + ut) * (wc + wE);
      fB_n = (vc + vn) * (vc + vn);
      fvw = (vc + vt) * (wc + wn);
      c_t = (wc + wt) * (wc + wt);
      sA[b][ty][tx] = fA_e;
      sUV[b][ty][tx] = fuv;
      sUW[b][ty][tx] = fuw;
      sB[b][ty][tx] = fB_n;
      sVW[b][ty][tx] = fvw;
    }
    __syncthreads();
    if (live) {
      // west fluxes: from the thread to the west, or formed here on the tile's first column
      double fA_w, fuv_w, fuw_w;
      const double uw = u[at(iw, j, k)];
      if (tx > 0) {
        fA_w = sA[b][ty][tx - 1];
        fuv_w = sUV[b][ty][tx - 1];
        fuw_w = sUW[b][ty][tx - 1];
      } else {
        fA_w = (uw + uc) * (uw + uc);
        fuv_w = (uw + u[at(iw, jn, k)]) * (v[at(iw, j, k)] + vc);
        fuw_w = (uw + U(u, iw, j, k + 1)) * (Wv(iw, j, k) + wc);
      }
      // south fluxes
      double fuv_s, fB_s, fvw_s;
      const double vs_ = v[at(i, js, k)];
      if (ty > 0) {
        fuv_s = sUV[b][ty - 1][tx];
        fB_s = sB[b][ty - 1][tx];
        fvw_s = sVW[b][ty - 1][tx];
      } else {
        fuv_s = (u[at(i, js, k)] + uc) * (vs_ + v[at(ie, js, k)]);
        fB_s = (vs_ + vc) * (vs_ + vc);
        fvw_s = (vs_ + U(v, i, js, k + 1)) * (Wv(i, js, k) + wc);
      }
      const double dzfi = g.dzfi[k], dzc_up = g.dzci[k], qdz = 0.25 * dzfi;
      const double uS = u[at(i, js, k)], vW = v[at(iw, j, k)];
      // second differences along x and y, z first differences (carried to the next plane)
      const double xx_u = fma(-2.0, uc, ue + uw), yy_u = fma(-2.0, uc, un + uS), gu_t = (ut - uc) * dzc_up;
      const double xx_v = fma(-2.0, vc, vE + vW), yy_v = fma(-2.0, vc, vn + vs_), gv_t = (vt - vc) * dzc_up;
      double r_u, r_v, r_w = 0.0, lap_u = 0.0, lap_v = 0.0, lap_w = 0.0, hw_t = 0.0;
      if (IMPL) {  // the Helmholtz right-hand side needs L u on its own
        lap_u = fma(dx2, xx_u, fma(dy2, yy_u, (gu_t - gu_b) * dzfi));
        lap_v = fma(dx2, xx_v, fma(dy2, yy_v, (gv_t - gv_b) * dzfi));
        r_u = -fma(qdx, fA_e - fA_w, fma(qdy, fuv - fuv_s, qdz * (fuw - fuw_b)));
        r_v = -fma(qdx, fuv - fuv_w, fma(qdy, fB_n - fB_s, qdz * (fvw - fvw_b)));
      } else {  // nu L u - A(u) as one chain, nu folded into the metric factors
        const double ndz = nu * dzfi;
        r_u = fma(ndx2, xx_u, fma(ndy2, yy_u, fma(ndz, gu_t - gu_b,
              fma(-qdx, fA_e - fA_w, fma(-qdy, fuv - fuv_s, -qdz * (fuw - fuw_b))))));
        r_v = fma(ndx2, xx_v, fma(ndy2, yy_v, fma(ndz, gv_t - gv_b,
              fma(-qdx, fuv - fuv_w, fma(-qdy, fB_n - fB_s, -qdz * (fvw - fvw_b))))));
      }
      // w at (i, j, k+1/2); the top wall face stays at rest
      if (k < g.nz - 1) {
        const double qdzc = 0.25 * dzc_up;
        const double xx_w = fma(-2.0, wc, wE + Wv(iw, j, k)), yy_w = fma(-2.0, wc, wn + Wv(i, js, k));
        hw_t = (wt - wc) * g.dzfi[k + 1];
        if (IMPL) {
          lap_w = fma(dx2, xx_w, fma(dy2, yy_w, (hw_t - hw_b) * dzc_up));
          r_w = -fma(qdx, fuw - fuw_w, fma(qdy, fvw - fvw_s, qdzc * (c_t - c_b)));
        } else {
          r_w = fma(ndx2, xx_w, fma(ndy2, yy_w, fma(nu * dzc_up, hw_t - hw_b,
                fma(-qdx, fuw - fuw_w, fma(-qdy, fvw - fvw_s, -qdzc * (c_t - c_b))))));
        }
      }
      // u* = u + dt (alpha r + beta r_prev - gamma G p): dt alpha, dt beta and -dt gamma / dx folded
      const double pc = p[c];
      const double dpx = p[at(ie, j, k)] - pc, dpy = p[at(i, jn, k)] - pc;
      const double dpz = (k < g.nz - 1) ? p[c + plane] - pc : 0.0;
      if (IMPL) {
        double su = fma(dga_x, dpx, fma(dta, r_u, uc)), sv = fma(dga_y, dpy, fma(dta, r_v, vc));
        double sw = fma(dtg * dzc_up, dpz, fma(dta, r_w, wc));
        if (beta != 0.0) {
          su = fma(dtb, ru[c], su);
          sv = fma(dtb, rv[c], sv);
          sw = fma(dtb, rw[c], sw);
        }
        us[c] = fma(sigma, su, -lap_u);
        vs[c] = fma(sigma, sv, -lap_v);
        ws[c] = (k < g.nz - 1) ? fma(sigma, sw, -lap_w) : 0.0;
      } else {
        double su = fma(dga_x, dpx, fma(dta, r_u, uc)), sv = fma(dga_y, dpy, fma(dta, r_v, vc));
        double sw = fma(dtg * dzc_up, dpz, fma(dta, r_w, wc));
        if (beta != 0.0) {
          su = fma(dtb, ru[c], su);
          sv = fma(dtb, rv[c], sv);
          sw = fma(dtb, rw[c], sw);
        }
        us[c] = su;
        vs[c] = sv;
        ws[c] = (k < g.nz - 1) ? sw : 0.0;
      }
      ru[c] = r_u;
      rv[c] = r_v;
      rw[c] = r_w;
      // carry the top quantities to the next plane's bottom
      fuw_b = fuw;
      fvw_b = fvw;
      c_b = c_t;
      gu_b = gu_t;
      gv_b = gv_t;
      hw_b = hw_t;
    }
    // no barrier here: the next plane writes the other buffer, and the plane after it reaches this
    // buffer only after every thread has passed the next plane's barrier, i.e. finished these reads
  }
}

// f = D(u) * scale (cell-centred divergence, Eq. poi_ns right-hand side with scale = 1/(gamma dt)).
// Adjoint use: the face field is first divided by its face weight (dzf for u and v, dzc for w).
__global__ void divergence_kernel(Chan g, const double* __restrict__ u, const double* __restrict__ v,
                                  const double* __restrict__ w, double* __restrict__ f, double scale_num,
                                  const double* __restrict__ dt_dev, double gamma, int weighted, DivArgs dv) {
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  const double scale = (dt_dev != nullptr) ? scale_num / (gamma * (*dt_dev)) : scale_num;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / ((size_t)g.nx * g.ny));
    if (!weighted) {  // the arithmetic the fused x pass repeats bit for bit
      f[c] = dv.at(scale, c, i, j, k);
      continue;
    }
    double uw = u[c] - u[g.id(i - 1, j, k)];
    double vw = v[c] - v[g.id(i, j - 1, k)];
    double wt = Wn(g, w, i, j, k), wb = Wn(g, w, i, j, k - 1);
    uw *= g.dzfi[k];
    vw *= g.dzfi[k];
    wt *= (k < g.nz - 1) ? 2.0 / (g.dzf[k] + g.dzf[k + 1]) : 0.0;
    wb *= (k > 0) ? 2.0 / (g.dzf[k - 1] + g.dzf[k]) : 0.0;
    f[c] = scale * (uw * g.dxi + vw * g.dyi + (wt - wb) * g.dzfi[k]);
  }
}

// u = u* - gamma dt G Phi (Eq. poi_ns correction), p += Phi when p != nullptr, and the dzf-weighted
// sum of the new u into *bulk.out (for the constant-flow-rate forcing; a reproducible block sum).  Adjoint use (weighted): the
// gradient is multiplied by the face weight.
// Crank-Nicolson diffusion (Eq. up_id_2): p += Phi + lcoef L_p Phi with lcoef = -gamma nu dt/2 and L_p
// the pressure Laplacian (periodic x, y; Neumann walls).
__global__ void correct_kernel(Chan g, const double* __restrict__ us, const double* __restrict__ vs,
                               const double* __restrict__ ws, const double* __restrict__ phi, double* __restrict__ u,
                               double* __restrict__ v, double* __restrict__ w, double* __restrict__ p, double gamma,
                               const double* __restrict__ dt_dev, int weighted, DetSum bulk, double lcoef) {
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  const double f = (dt_dev != nullptr) ? gamma * (*dt_dev) : 1.0;
  double acc = 0.0;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / ((size_t)g.nx * g.ny));
    const double pc = phi[c];
    double gx = (phi[g.id(i + 1, j, k)] - pc) * g.dxi;
    double gy = (phi[g.id(i, j + 1, k)] - pc) * g.dyi;
    double gz = (k < g.nz - 1) ? (phi[g.id(i, j, k + 1)] - pc) * g.dzci[k] : 0.0;
    if (weighted) {
      gx *= g.dzf[k];
      gy *= g.dzf[k];
      gz *= (k < g.nz - 1) ? 0.5 * (g.dzf[k] + g.dzf[k + 1]) : 0.0;
    }
    const double un = us[c] - f * gx;
    u[c] = un;
    v[c] = vs[c] - f * gy;
    w[c] = (k < g.nz - 1) ? ws[c] - f * gz : 0.0;
    if (p != nullptr) {
      double dp = pc;
      if (lcoef != 0.0) {
        const double pxm = phi[g.id(i - 1, j, k)], pxp = phi[g.id(i + 1, j, k)];
        const double pym = phi[g.id(i, j - 1, k)], pyp = phi[g.id(i, j + 1, k)];
        const double fup = (k < g.nz - 1) ? (phi[g.id(i, j, k + 1)] - pc) * g.dzci[k] : 0.0;
        const double fdn = (k > 0) ? (pc - phi[g.id(i, j, k - 1)]) * g.dzci[k - 1] : 0.0;
        const double lap = (pxm - 2 * pc + pxp) * g.dxi * g.dxi + (pym - 2 * pc + pyp) * g.dyi * g.dyi +
                           (fup - fdn) * g.dzfi[k];
        dp = fma(lcoef, lap, pc);
      }
      p[c] += dp;
    }
    acc += g.dzf[k] * un;
  }
  if (bulk.out != nullptr) det_sum_finish(block_sum_d(acc), bulk);
}

// u += ubulk - <u>_V with <u>_V = bulk / (Nx Ny sum dzf)
__global__ void forcing_kernel(Chan g, double* __restrict__ u, const double* __restrict__ bulk, double inv_vol,
                               double ubulk) {
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  const double shift = ubulk - (*bulk) * inv_vol;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x)
    u[c] += shift;
}

// largest inverse advective time scale over all cells (chkdt listing, y and z rows by symmetry),
// reduced on the device: block maximum, then one atomic max on the bit pattern (non-negative doubles
// order like their bits).
// The largest inverse advective time scale of cell (i, j, k) (Eq. dt and its chkdt rows; the y and z
// rows follow the x row by symmetry), in FP64; the 1/4 of the four-point averages is folded into the
// metric factors (fewer FP64 operations).
__device__ __forceinline__ double dti_cell(const Chan& g, const double* __restrict__ u, const double* __restrict__ v,
                                           const double* __restrict__ w, size_t c, int i, int j, int k) {
  const double qdx = 0.25 * g.dxi, qdy = 0.25 * g.dyi, qdz = 0.25 * g.dzfi[k];
  const double vx = fabs(v[c] + v[g.id(i, j - 1, k)] + v[g.id(i + 1, j, k)] + v[g.id(i + 1, j - 1, k)]);
  const double wx = fabs(Wn(g, w, i, j, k) + Wn(g, w, i, j, k - 1) + Wn(g, w, i + 1, j, k) + Wn(g, w, i + 1, j, k - 1));
  const double dtix = fma(fabs(u[c]), g.dxi, fma(vx, qdy, wx * qdz));
  const double uy = fabs(u[c] + u[g.id(i - 1, j, k)] + u[g.id(i, j + 1, k)] + u[g.id(i - 1, j + 1, k)]);
  const double wy = fabs(Wn(g, w, i, j, k) + Wn(g, w, i, j, k - 1) + Wn(g, w, i, j + 1, k) + Wn(g, w, i, j + 1, k - 1));
  const double dtiy = fma(uy, qdx, fma(fabs(v[c]), g.dyi, wy * qdz));
  const double uz = fabs(u[c] + u[g.id(i - 1, j, k)] + Ut(g, u, i, j, k + 1) + Ut(g, u, i - 1, j, k + 1));
  const double vz = fabs(v[c] + v[g.id(i, j - 1, k)] + Ut(g, v, i, j, k + 1) + Ut(g, v, i, j - 1, k + 1));
  const double dtiz = fma(uz, qdx, fma(vz, qdy, fabs(Wn(g, w, i, j, k)) * g.dzci[k]));
  return fmax(dtix, fmax(dtiy, dtiz));
}

__global__ void chkdt_kernel(Chan g, const double* __restrict__ u, const double* __restrict__ v,
                             const double* __restrict__ w, unsigned long long* dti_bits) {
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  double dti = 0.0;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / ((size_t)g.nx * g.ny));
    dti = fmax(dti, dti_cell(g, u, v, w, c, i, j, k));
  }
  for (int o = 16; o > 0; o >>= 1) dti = fmax(dti, __shfl_xor_sync(0xffffffffu, dti, o));
  if ((threadIdx.x & 31) == 0) atomicMax(dti_bits, (unsigned long long)__double_as_longlong(dti));
}

// dt = cfl * min(sqrt(3)/dti, 1.65 dl^2/nu) (Eq. dt), or the fixed value when dt_fixed > 0
__global__ void dt_kernel(const unsigned long long* dti_bits, double* dt_dev, double cfl, double nu, double dl,
                          double dt_fixed) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (dt_fixed > 0) {
    *dt_dev = dt_fixed;
    return;
  }
  const double dti = __longlong_as_double((long long)*dti_bits);
  double dt = 1.65 * dl * dl / nu;
  if (dti > 0) dt = fmin(dt, 1.7320508075688772935 / dti);
  *dt_dev = cfl * dt;
}

static Chan chan(const cans_plan_s* P) {
  Chan g;
  g.nx = P->n[0];
  g.ny = P->n[1];
  g.nz = P->n[2];
  g.dxi = P->n[0] / P->len[0];
  g.dyi = P->n[1] / P->len[1];
  g.dzf = P->dzf_d;
  g.dzfi = P->dzfi_d;
  g.dzci = P->dzci_d;
  return g;
}

static int grid_for(size_t N) {
  size_t b = (N + 255) / 256;
  return (int)std::min<size_t>(b, (size_t)148 * 16);
}

cudaError_t launch_momentum(const cans_plan_s* P, const double* u, const double* v, const double* w, const double* p,
                            double* ru, double* rv, double* rw, double* us, double* vs, double* ws, double nu,
                            double alpha, double beta, double gamma, const double* dt_dev, cudaStream_t st,
                            double sigma) {
  const Chan g = chan(P);
  const dim3 grid((g.nx + MX - 1) / MX, (g.ny + MY - 1) / MY, (g.nz + MZ - 1) / MZ), block(MX, MY);
  if (sigma != 0.0)
    momentum_flux_kernel<true><<<grid, block, 0, st>>>(g, u, v, w, p, ru, rv, rw, us, vs, ws, nu, alpha, beta, gamma,
                                                       dt_dev, sigma);
  else
    momentum_flux_kernel<false><<<grid, block, 0, st>>>(g, u, v, w, p, ru, rv, rw, us, vs, ws, nu, alpha, beta, gamma,
                                                        dt_dev, sigma);
  return cudaGetLastError();
}

cudaError_t launch_divergence(const cans_plan_s* P, const double* u, const double* v, const double* w, double* f,
                              double scale_num, const double* dt_dev, double gamma, int weighted, cudaStream_t st) {
  const Chan g = chan(P);
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  divergence_kernel<<<grid_for(N), 256, 0, st>>>(g, u, v, w, f, scale_num, dt_dev, gamma, weighted,
                                                 div_args(P, u, v, w, f, scale_num, dt_dev, gamma));
  return cudaGetLastError();
}

DivArgs div_args(const cans_plan_s* P, const double* u, const double* v, const double* w, double* fout, double num,
                 const double* dt, double gamma) {
  const Chan g = chan(P);
  DivArgs d;
  d.u = u;
  d.v = v;
  d.w = w;
  d.fout = fout;
  d.dzfi = g.dzfi;
  d.dt = dt;
  d.num = num;
  d.gamma = gamma;
  d.dxi = g.dxi;
  d.dyi = g.dyi;
  d.nx = g.nx;
  d.ny = g.ny;
  d.nz = g.nz;
  return d;
}

cudaError_t launch_correct(const cans_plan_s* P, const double* us, const double* vs, const double* ws,
                           const double* phi, double* u, double* v, double* w, double* p, double gamma,
                           const double* dt_dev, int weighted, double* bulk, cudaStream_t st, double lcoef) {
  const Chan g = chan(P);
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  const int grid = grid_for(N);
  if ((size_t)grid > P->dsum_nslots) return cudaErrorInvalidConfiguration;
  correct_kernel<<<grid, 256, 0, st>>>(g, us, vs, ws, phi, u, v, w, p, gamma, dt_dev, weighted, plan_sum(P, bulk),
                                       lcoef);
  return cudaGetLastError();
}

cudaError_t launch_forcing(const cans_plan_s* P, double* u, const double* bulk, double ubulk, cudaStream_t st) {
  const Chan g = chan(P);
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  double lz = 0;
  for (int k = 0; k < g.nz; ++k) lz += P->dzf_h[k];
  forcing_kernel<<<grid_for(N), 256, 0, st>>>(g, u, bulk, 1.0 / ((double)g.nx * g.ny * lz), ubulk);
  return cudaGetLastError();
}

cudaError_t launch_chkdt(const cans_plan_s* P, const double* u, const double* v, const double* w,
                         unsigned long long* dti_bits, double* dt_dev, double cfl, double nu, double dt_fixed,
                         cudaStream_t st) {
  const Chan g = chan(P);
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  cudaError_t e = cudaMemsetAsync(dti_bits, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  if (dt_fixed <= 0) chkdt_kernel<<<grid_for(N), 256, 0, st>>>(g, u, v, w, dti_bits);
  double dl = std::min(P->len[0] / P->n[0], P->len[1] / P->n[1]);
  for (int k = 0; k < g.nz; ++k) dl = std::min(dl, P->dzf_h[k]);
  dt_kernel<<<1, 32, 0, st>>>(dti_bits, dt_dev, cfl, nu, dl, dt_fixed);
  return cudaGetLastError();
}

}  // namespace cans

// ------------------------------------------------------------------------------------------------
// C ABI: one RK3 step, the projection and its adjoint
// ------------------------------------------------------------------------------------------------
using namespace cans;

namespace {

// NVTX range of one RK3 substage (host timeline of its enqueued work; a no-op without a tool)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

const double RK_ALPHA[3] = {8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0};
const double RK_BETA[3] = {0.0, -17.0 / 60.0, -5.0 / 12.0};

bool is_channel(const cans_plan_s* P) { return P->bc[0] == BC_P && P->bc[1] == BC_P && P->bc[2] == BC_NN; }

size_t a256(size_t b) { return (b + 255) & ~size_t(255); }

#define RK_CK(...)                                 \
  do {                                             \
    cudaError_t e_ = (__VA_ARGS__);                \
    if (e_ != cudaSuccess) return CANS_ERR_CUDA;   \
  } while (0)

}  // namespace

extern "C" {

int cans_rk3_workspace_size(cans_plan_t P, size_t* bytes) {
  if (!P || !bytes) return CANS_ERR_ARG;
  const size_t N = (size_t)P->n[0] * P->n[1] * P->n[2];
  size_t pws = 0;
  cans_poisson_workspace_size(P, &pws);
  *bytes = 8 * a256(N * sizeof(double)) + 256 + a256(pws);
  return CANS_OK;
}

int cans_rk3_step(cans_plan_t P, double* u, double* v, double* w, double* p, const cans_rk3_params* prm,
                  double* dt_dev, void* workspace, void* cuda_stream) {
  if (!P || !u || !v || !w || !p || !prm || !workspace) return CANS_ERR_ARG;
  if (!is_channel(P)) return CANS_ERR_UNSUPPORTED;
  if (!(prm->nu > 0) || !(prm->cfl > 0)) return CANS_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(workspace) & 255) return CANS_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const size_t N = (size_t)P->n[0] * P->n[1] * P->n[2];
  const size_t fb = a256(N * sizeof(double));
  unsigned char* base = static_cast<unsigned char*>(workspace);
  double* us = reinterpret_cast<double*>(base + 0 * fb);
  double* vs = reinterpret_cast<double*>(base + 1 * fb);
  double* ws = reinterpret_cast<double*>(base + 2 * fb);
  double* ru = reinterpret_cast<double*>(base + 3 * fb);
  double* rv = reinterpret_cast<double*>(base + 4 * fb);
  double* rw = reinterpret_cast<double*>(base + 5 * fb);
  double* f = reinterpret_cast<double*>(base + 6 * fb);
  double* phi = reinterpret_cast<double*>(base + 7 * fb);
  double* small = reinterpret_cast<double*>(base + 8 * fb);  // [0] dt, [1] bulk sum, [2] dti bits
  void* pws = base + 8 * fb + 256;
  double* dt = dt_dev ? dt_dev : small;
  {
    PassTimer tm(P, CANS_PASS_CHKDT, st);
    RK_CK(launch_chkdt(P, u, v, w, reinterpret_cast<unsigned long long*>(small + 2), dt, prm->cfl, prm->nu, prm->dt,
                       st));
  }
  for (int s = 0; s < 3; ++s) {
    NvtxRange substage(s == 0 ? "rk3_substage_1" : (s == 1 ? "rk3_substage_2" : "rk3_substage_3"));
    const double a = RK_ALPHA[s], b = RK_BETA[s], g = a + b;
    {
      PassTimer tm(P, CANS_PASS_MOMENTUM, st);
      RK_CK(launch_momentum(P, u, v, w, p, ru, rv, rw, us, vs, ws, prm->nu, a, b, g, dt, st));
    }
    // Eq. poi_ns: the divergence as its own kernel, then the solve.  (Forming the divergence inside the
    // solve's first x pass, cans_poisson_solve_divergence, saves its 16 B/pt of traffic, but both
    // forms are bound by the divergence's FP64 operations on this GPU, and the separate kernel hides
    // their latency better: measured 0.54 ms faster per step at 512 x 256 x 192.)
    {
      PassTimer tm(P, CANS_PASS_DIVERGENCE, st);
      RK_CK(launch_divergence(P, us, vs, ws, f, 1.0, dt, g, 0, st));
    }
    int rc = cans_poisson_solve(P, f, phi, pws, cuda_stream, nullptr);
    if (rc != CANS_OK) return rc;
    double* bulk = prm->forcing ? small + 1 : nullptr;
    {
      PassTimer tm(P, CANS_PASS_CORRECT, st);
      RK_CK(launch_correct(P, us, vs, ws, phi, u, v, w, p, g, dt, 0, bulk, st));
    }
    if (bulk) {
      PassTimer tm(P, CANS_PASS_FORCING, st);
      RK_CK(launch_forcing(P, u, bulk, prm->ubulk, st));
    }
  }
  return CANS_OK;
}

// The velocity plans of the implicit step must describe the pressure plan's grid: (P, P, DD) with
// the same Nx, Ny, lengths; uv on the cell grid of the same dzf, w on its interior faces.
static bool implicit_plans_match(const cans_plan_s* P, const cans_plan_s* U, const cans_plan_s* W) {
  if (!U || !W) return false;
  const int nz = P->n[2];
  for (const cans_plan_s* Q : {U, W}) {
    if (Q->n[0] != P->n[0] || Q->n[1] != P->n[1] || Q->len[0] != P->len[0] || Q->len[1] != P->len[1]) return false;
    if (Q->bc[0] != BC_P || Q->bc[1] != BC_P || Q->bc[2] != BC_DD) return false;
  }
  if (U->opts.z_grid != 0 || U->n[2] != nz || W->opts.z_grid != 1 || W->nz_cells != nz) return false;
  for (int k = 0; k < nz; ++k)
    if (std::fabs(U->dzf_h[k] - P->dzf_h[k]) > 1e-14 * P->dzf_h[k]) return false;
  for (int k = 0; k + 1 < nz; ++k) {
    const double mid = 0.5 * (P->dzf_h[k] + P->dzf_h[k + 1]);
    if (std::fabs(W->dzf_h[k] - mid) > 1e-14 * mid) return false;
  }
  return true;
}

int cans_rk3_implicit_workspace_size(cans_plan_t P, cans_plan_t U, cans_plan_t W, size_t* bytes) {
  if (!P || !U || !W || !bytes) return CANS_ERR_ARG;
  const size_t N = (size_t)P->n[0] * P->n[1] * P->n[2];
  size_t pws = 0, b = 0;
  for (const cans_plan_s* Q : {P, U, W}) {
    cans_poisson_workspace_size(const_cast<cans_plan_t>(Q), &b);
    pws = std::max(pws, b);
  }
  *bytes = 10 * a256(N * sizeof(double)) + 256 + a256(pws);
  return CANS_OK;
}

int cans_rk3_step_implicit(cans_plan_t P, cans_plan_t U, cans_plan_t W, double* u, double* v, double* w, double* p,
                           const cans_rk3_params* prm, double* dt_dev, void* workspace, void* cuda_stream) {
  if (!P || !u || !v || !w || !p || !prm || !workspace) return CANS_ERR_ARG;
  if (!is_channel(P)) return CANS_ERR_UNSUPPORTED;
  if (!implicit_plans_match(P, U, W)) return CANS_ERR_ARG;
  if (!(prm->nu > 0) || !(prm->dt > 0) || !std::isfinite(prm->dt)) return CANS_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(workspace) & 255) return CANS_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const size_t N = (size_t)P->n[0] * P->n[1] * P->n[2];
  const size_t fb = a256(N * sizeof(double));
  unsigned char* base = static_cast<unsigned char*>(workspace);
  double* F[10];
  for (int q = 0; q < 10; ++q) F[q] = reinterpret_cast<double*>(base + q * fb);
  double *us = F[0], *vs = F[1], *ws = F[2], *ru = F[3], *rv = F[4], *rw = F[5], *fu = F[6], *fv = F[7], *fw = F[8];
  double* phi = F[9];
  double* f = fu;  // the divergence reuses the first Helmholtz right-hand side
  double* small = reinterpret_cast<double*>(base + 10 * fb);  // [0] dt, [1] bulk sum, [2] dti bits
  void* pws = base + 10 * fb + 256;
  double* dt = dt_dev ? dt_dev : small;
  {
    PassTimer tm(P, CANS_PASS_CHKDT, st);
    RK_CK(launch_chkdt(P, u, v, w, reinterpret_cast<unsigned long long*>(small + 2), dt, prm->cfl, prm->nu, prm->dt,
                       st));
  }
  for (int s = 0; s < 3; ++s) {
    NvtxRange substage(s == 0 ? "rk3_implicit_substage_1" : (s == 1 ? "rk3_implicit_substage_2" : "rk3_implicit_substage_3"));
    const double a = RK_ALPHA[s], b = RK_BETA[s], g = a + b;
    const double h = g * prm->nu * prm->dt / 2, sigma = -1.0 / h;
    {
      PassTimer tm(P, CANS_PASS_MOMENTUM, st);
      RK_CK(launch_momentum(P, u, v, w, p, ru, rv, rw, fu, fv, fw, prm->nu, a, b, g, dt, st, sigma));
    }
    int rc = cans_helmholtz_solve(U, fu, us, sigma, pws, cuda_stream, nullptr);
    if (rc == CANS_OK) rc = cans_helmholtz_solve(U, fv, vs, sigma, pws, cuda_stream, nullptr);
    if (rc == CANS_OK) rc = cans_helmholtz_solve(W, fw, ws, sigma, pws, cuda_stream, nullptr);
    if (rc != CANS_OK) return rc;
    {
      PassTimer tm(P, CANS_PASS_DIVERGENCE, st);
      RK_CK(cudaMemsetAsync(ws + (size_t)P->n[0] * P->n[1] * (P->n[2] - 1), 0,
                            sizeof(double) * P->n[0] * P->n[1], st));  // the top wall face
      RK_CK(launch_divergence(P, us, vs, ws, f, 1.0, dt, g, 0, st));
    }
    rc = cans_poisson_solve(P, f, phi, pws, cuda_stream, nullptr);
    if (rc != CANS_OK) return rc;
    double* bulk = prm->forcing ? small + 1 : nullptr;
    {
      PassTimer tm(P, CANS_PASS_CORRECT, st);
      RK_CK(launch_correct(P, us, vs, ws, phi, u, v, w, p, g, dt, 0, bulk, st, -h));
    }
    if (bulk) {
      PassTimer tm(P, CANS_PASS_FORCING, st);
      RK_CK(launch_forcing(P, u, bulk, prm->ubulk, st));
    }
  }
  return CANS_OK;
}

int cans_project_workspace_size(cans_plan_t P, size_t* bytes) {
  if (!P || !bytes) return CANS_ERR_ARG;
  const size_t N = (size_t)P->n[0] * P->n[1] * P->n[2];
  size_t pws = 0;
  cans_poisson_workspace_size(P, &pws);
  *bytes = 2 * a256(N * sizeof(double)) + a256(pws);
  return CANS_OK;
}

static int project_impl(cans_plan_t P, double* u, double* v, double* w, void* workspace, void* cuda_stream,
                        int adjoint) {
  if (!P || !u || !v || !w || !workspace) return CANS_ERR_ARG;
  if (!is_channel(P)) return CANS_ERR_UNSUPPORTED;
  if (reinterpret_cast<uintptr_t>(workspace) & 255) return CANS_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const size_t N = (size_t)P->n[0] * P->n[1] * P->n[2];
  const size_t fb = a256(N * sizeof(double));
  unsigned char* base = static_cast<unsigned char*>(workspace);
  double* f = reinterpret_cast<double*>(base);
  double* phi = reinterpret_cast<double*>(base + fb);
  void* pws = base + 2 * fb;
  {
    PassTimer tm(P, CANS_PASS_DIVERGENCE, st);
    RK_CK(launch_divergence(P, u, v, w, f, 1.0, nullptr, 1.0, adjoint, st));
  }
  int rc = cans_poisson_solve(P, f, phi, pws, cuda_stream, nullptr);
  if (rc != CANS_OK) return rc;
  PassTimer tm(P, CANS_PASS_CORRECT, st);
  RK_CK(launch_correct(P, u, v, w, phi, u, v, w, nullptr, 1.0, nullptr, adjoint, nullptr, st));
  return CANS_OK;
}

int cans_project(cans_plan_t P, double* u, double* v, double* w, void* workspace, void* cuda_stream) {
  return project_impl(P, u, v, w, workspace, cuda_stream, 0);
}

int cans_project_adjoint(cans_plan_t P, double* u, double* v, double* w, void* workspace, void* cuda_stream) {
  return project_impl(P, u, v, w, workspace, cuda_stream, 1);
}

}  // extern "C"
