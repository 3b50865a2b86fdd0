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
//   u* = u + dt (alpha rhs + beta rhs_prev - gamma G p).  rhs replaces rhs_prev in place.
// IMPL (Crank-Nicolson diffusion, Eq. up_id and Eq. up_id_2): rhs = A(u) alone, and us receives the
// right-hand side of the Helmholtz problem (L + sigma) u* = sigma (u** - gamma nu dt/2 L u), sigma =
// -2/(gamma nu dt), which is sigma (u + dt (alpha A + beta A_prev - gamma G p)) - L u.
template <bool IMPL>
__global__ void momentum_kernel(Chan g, const double* __restrict__ u, const double* __restrict__ v,
                                const double* __restrict__ w, const double* __restrict__ p, double* __restrict__ ru,
                                double* __restrict__ rv, double* __restrict__ rw, double* __restrict__ us,
                                double* __restrict__ vs, double* __restrict__ ws, double nu, double alpha, double beta,
                                double gamma, const double* __restrict__ dt_dev, double sigma) {
  // The same discrete operator as written term by term (two-point averages, products, differences),
  // arranged for fewer FP64 operations (B300 issues FP64 at 1/64 of FP32): the 1/2 x 1/2 factors of
  // the averaged products and 1/dx^2 are folded into constants, (ue^2 - uw^2) is formed as
  // (u_e - u_w)(u_e + 2 u_c + u_w), and sums of products use FMA.
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  const double dt = *dt_dev;
  const double qdx = 0.25 * g.dxi, qdy = 0.25 * g.dyi, dx2 = g.dxi * g.dxi, dy2 = g.dyi * g.dyi;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / ((size_t)g.nx * g.ny));
    const double qdz = 0.25 * g.dzfi[k], dzfi = g.dzfi[k], dzc_up = g.dzci[k], dzc_dn = dzc_inv_below(g, k);
    const double uc = u[c], vc = v[c];
    double r_u, r_v, r_w, l_u, l_v, l_w = 0.0;
    {  // u at (i+1/2, j, k)
      const double ue = u[g.id(i + 1, j, k)], uw = u[g.id(i - 1, j, k)];
      const double un = u[g.id(i, j + 1, k)], uS = u[g.id(i, j - 1, k)];
      const double ut = Ut(g, u, i, j, k + 1), ub = Ut(g, u, i, j, k - 1);
      const double ax = (ue - uw) * fma(2.0, uc, ue + uw);
      const double ay = fma(-(uS + uc), v[g.id(i, j - 1, k)] + v[g.id(i + 1, j - 1, k)],
                            (uc + un) * (vc + v[g.id(i + 1, j, k)]));
      const double az = fma(-(ub + uc), Wn(g, w, i, j, k - 1) + Wn(g, w, i + 1, j, k - 1),
                            (uc + ut) * (Wn(g, w, i, j, k) + Wn(g, w, i + 1, j, k)));
      const double adv = fma(qdx, ax, fma(qdy, ay, qdz * az));
      const double lz = fma(ut - uc, dzc_up, -(uc - ub) * dzc_dn) * dzfi;
      const double lap = fma(dx2, fma(-2.0, uc, ue + uw), fma(dy2, fma(-2.0, uc, un + uS), lz));
      r_u = IMPL ? -adv : fma(nu, lap, -adv);
      l_u = lap;
    }
    {  // v at (i, j+1/2, k)
      const double ve = v[g.id(i + 1, j, k)], vw = v[g.id(i - 1, j, k)];
      const double vn = v[g.id(i, j + 1, k)], vS = v[g.id(i, j - 1, k)];
      const double vt = Ut(g, v, i, j, k + 1), vb = Ut(g, v, i, j, k - 1);
      const double ax = fma(-(vw + vc), u[g.id(i - 1, j, k)] + u[g.id(i - 1, j + 1, k)],
                            (vc + ve) * (uc + u[g.id(i, j + 1, k)]));
      const double ay = (vn - vS) * fma(2.0, vc, vn + vS);
      const double az = fma(-(vb + vc), Wn(g, w, i, j, k - 1) + Wn(g, w, i, j + 1, k - 1),
                            (vc + vt) * (Wn(g, w, i, j, k) + Wn(g, w, i, j + 1, k)));
      const double adv = fma(qdx, ax, fma(qdy, ay, qdz * az));
      const double lz = fma(vt - vc, dzc_up, -(vc - vb) * dzc_dn) * dzfi;
      const double lap = fma(dx2, fma(-2.0, vc, ve + vw), fma(dy2, fma(-2.0, vc, vn + vS), lz));
      r_v = IMPL ? -adv : fma(nu, lap, -adv);
      l_v = lap;
    }
    if (k == g.nz - 1) {
      r_w = 0.0;
    } else {  // w at (i, j, k+1/2)
      const double wc = w[c];
      const double we = Wn(g, w, i + 1, j, k), ww = Wn(g, w, i - 1, j, k);
      const double wn = Wn(g, w, i, j + 1, k), wS = Wn(g, w, i, j - 1, k);
      const double wt = Wn(g, w, i, j, k + 1), wb = Wn(g, w, i, j, k - 1);
      const double qdzc = 0.25 * dzc_up;
      const double ax = fma(-(ww + wc), u[g.id(i - 1, j, k)] + u[g.id(i - 1, j, k + 1)],
                            (wc + we) * (uc + u[g.id(i, j, k + 1)]));
      const double ay = fma(-(wS + wc), v[g.id(i, j - 1, k)] + v[g.id(i, j - 1, k + 1)],
                            (wc + wn) * (vc + v[g.id(i, j, k + 1)]));
      const double az = (wt - wb) * fma(2.0, wc, wt + wb);
      const double adv = fma(qdx, ax, fma(qdy, ay, qdzc * az));
      const double lz = fma(wt - wc, g.dzfi[k + 1], -(wc - wb) * dzfi) * dzc_up;
      const double lap = fma(dx2, fma(-2.0, wc, we + ww), fma(dy2, fma(-2.0, wc, wn + wS), lz));
      r_w = IMPL ? -adv : fma(nu, lap, -adv);
      l_w = lap;
    }
    const double pc = p[c];
    const double gx = (p[g.id(i + 1, j, k)] - pc) * g.dxi;
    const double gy = (p[g.id(i, j + 1, k)] - pc) * g.dyi;
    const double gz = (k < g.nz - 1) ? (p[g.id(i, j, k + 1)] - pc) * dzc_up : 0.0;
    double su = alpha * r_u, sv = alpha * r_v, sw = alpha * r_w;
    if (beta != 0.0) {
      su = fma(beta, ru[c], su);
      sv = fma(beta, rv[c], sv);
      sw = fma(beta, rw[c], sw);
    }
    if (IMPL) {
      us[c] = fma(sigma, fma(dt, fma(-gamma, gx, su), uc), -l_u);
      vs[c] = fma(sigma, fma(dt, fma(-gamma, gy, sv), vc), -l_v);
      ws[c] = (k < g.nz - 1) ? fma(sigma, fma(dt, fma(-gamma, gz, sw), w[c]), -l_w) : 0.0;
    } else {
      us[c] = fma(dt, fma(-gamma, gx, su), uc);
      vs[c] = fma(dt, fma(-gamma, gy, sv), vc);
      ws[c] = (k < g.nz - 1) ? fma(dt, fma(-gamma, gz, sw), w[c]) : 0.0;
    }
    ru[c] = r_u;
    rv[c] = r_v;
    rw[c] = r_w;
  }
}

// f = D(u) * scale (cell-centred divergence, Eq. poi_ns right-hand side with scale = 1/(gamma dt)).
// Adjoint use: the face field is first divided by its face weight (dzf for u and v, dzc for w).
__global__ void divergence_kernel(Chan g, const double* __restrict__ u, const double* __restrict__ v,
                                  const double* __restrict__ w, double* __restrict__ f, double scale_num,
                                  const double* __restrict__ dt_dev, double gamma, int weighted) {
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  const double scale = (dt_dev != nullptr) ? scale_num / (gamma * (*dt_dev)) : scale_num;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / ((size_t)g.nx * g.ny));
    double uw = u[c] - u[g.id(i - 1, j, k)];
    double vw = v[c] - v[g.id(i, j - 1, k)];
    double wt = Wn(g, w, i, j, k), wb = Wn(g, w, i, j, k - 1);
    if (weighted) {
      uw *= g.dzfi[k];
      vw *= g.dzfi[k];
      wt *= (k < g.nz - 1) ? 2.0 / (g.dzf[k] + g.dzf[k + 1]) : 0.0;
      wb *= (k > 0) ? 2.0 / (g.dzf[k - 1] + g.dzf[k]) : 0.0;
    }
    f[c] = scale * (uw * g.dxi + vw * g.dyi + (wt - wb) * g.dzfi[k]);
  }
}

// u = u* - gamma dt G Phi (Eq. poi_ns correction), p += Phi when p != nullptr, and the dzf-weighted
// sum of the new u into *bulk (for the constant-flow-rate forcing).  Adjoint use (weighted): the
// gradient is multiplied by the face weight.
// Crank-Nicolson diffusion (Eq. up_id_2): p += Phi + lcoef L_p Phi with lcoef = -gamma nu dt/2 and L_p
// the pressure Laplacian (periodic x, y; Neumann walls).
__global__ void correct_kernel(Chan g, const double* __restrict__ us, const double* __restrict__ vs,
                               const double* __restrict__ ws, const double* __restrict__ phi, double* __restrict__ u,
                               double* __restrict__ v, double* __restrict__ w, double* __restrict__ p, double gamma,
                               const double* __restrict__ dt_dev, int weighted, double* bulk, double lcoef) {
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
  if (bulk != nullptr) {
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(bulk, acc);
  }
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
__global__ void chkdt_kernel(Chan g, const double* __restrict__ u, const double* __restrict__ v,
                             const double* __restrict__ w, unsigned long long* dti_bits) {
  // the 1/4 of the four-point averages folded into the metric factors (fewer FP64 operations)
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  const double qdx = 0.25 * g.dxi, qdy = 0.25 * g.dyi;
  double dti = 0.0;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / ((size_t)g.nx * g.ny));
    const double qdz = 0.25 * g.dzfi[k];
    const double vx = fabs(v[c] + v[g.id(i, j - 1, k)] + v[g.id(i + 1, j, k)] + v[g.id(i + 1, j - 1, k)]);
    const double wx = fabs(Wn(g, w, i, j, k) + Wn(g, w, i, j, k - 1) + Wn(g, w, i + 1, j, k) + Wn(g, w, i + 1, j, k - 1));
    const double dtix = fma(fabs(u[c]), g.dxi, fma(vx, qdy, wx * qdz));
    const double uy = fabs(u[c] + u[g.id(i - 1, j, k)] + u[g.id(i, j + 1, k)] + u[g.id(i - 1, j + 1, k)]);
    const double wy = fabs(Wn(g, w, i, j, k) + Wn(g, w, i, j, k - 1) + Wn(g, w, i, j + 1, k) + Wn(g, w, i, j + 1, k - 1));
    const double dtiy = fma(uy, qdx, fma(fabs(v[c]), g.dyi, wy * qdz));
    const double uz = fabs(u[c] + u[g.id(i - 1, j, k)] + Ut(g, u, i, j, k + 1) + Ut(g, u, i - 1, j, k + 1));
    const double vz = fabs(v[c] + v[g.id(i, j - 1, k)] + Ut(g, v, i, j, k + 1) + Ut(g, v, i, j - 1, k + 1));
    const double dtiz = fma(uz, qdx, fma(vz, qdy, fabs(Wn(g, w, i, j, k)) * g.dzci[k]));
    dti = fmax(dti, fmax(dtix, fmax(dtiy, dtiz)));
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
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  if (sigma != 0.0)
    momentum_kernel<true><<<grid_for(N), 256, 0, st>>>(g, u, v, w, p, ru, rv, rw, us, vs, ws, nu, alpha, beta, gamma,
                                                       dt_dev, sigma);
  else
    momentum_kernel<false><<<grid_for(N), 256, 0, st>>>(g, u, v, w, p, ru, rv, rw, us, vs, ws, nu, alpha, beta, gamma,
                                                        dt_dev, 0.0);
  return cudaGetLastError();
}

cudaError_t launch_divergence(const cans_plan_s* P, const double* u, const double* v, const double* w, double* f,
                              double scale_num, const double* dt_dev, double gamma, int weighted, cudaStream_t st) {
  const Chan g = chan(P);
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  divergence_kernel<<<grid_for(N), 256, 0, st>>>(g, u, v, w, f, scale_num, dt_dev, gamma, weighted);
  return cudaGetLastError();
}

cudaError_t launch_correct(const cans_plan_s* P, const double* us, const double* vs, const double* ws,
                           const double* phi, double* u, double* v, double* w, double* p, double gamma,
                           const double* dt_dev, int weighted, double* bulk, cudaStream_t st, double lcoef) {
  const Chan g = chan(P);
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  correct_kernel<<<grid_for(N), 256, 0, st>>>(g, us, vs, ws, phi, u, v, w, p, gamma, dt_dev, weighted, bulk, lcoef);
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
    {
      PassTimer tm(P, CANS_PASS_DIVERGENCE, st);
      RK_CK(launch_divergence(P, us, vs, ws, f, 1.0, dt, g, 0, st));
    }
    int rc = cans_poisson_solve(P, f, phi, pws, cuda_stream, nullptr);
    if (rc != CANS_OK) return rc;
    double* bulk = prm->forcing ? small + 1 : nullptr;
    {
      PassTimer tm(P, CANS_PASS_CORRECT, st);
      if (bulk) RK_CK(cudaMemsetAsync(bulk, 0, sizeof(double), st));
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
      if (bulk) RK_CK(cudaMemsetAsync(bulk, 0, sizeof(double), st));
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
