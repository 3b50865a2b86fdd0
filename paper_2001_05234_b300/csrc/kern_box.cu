// The fractional step (Eq. up, Eq. poi_ns, the correction and p += Phi; Eq. dt) in a box whose every
// direction is periodic or bounded by no-slip walls, with an optional lid: the top z wall moving
// along x (lid-driven cavity: walls everywhere; square duct: x periodic; channel: z walls; decaying
// Taylor-Green vortex: periodic everywhere).  Marker-and-cell arrays as the channel step: u, v, w on
// the x-, y-, z-faces (index i is the face between cells i and i+1), p at cell centres.
//   * a velocity component normal to a walled direction is zero on both wall faces (the high one is
//     its last stored face, kept at 0);
//   * a tangential component beyond a wall takes the ghost 2 U_wall - (value in the wall cell), with
//     U_wall = lid for u at the top z wall and 0 otherwise; a corner ghost crosses x, then y, then z;
//   * the pressure is Neumann at walls (the plan's CANS_BC_NN), periodic elsewhere (CANS_BC_P).
// FP64 throughout, one thread per cell; the walls are compile-time so that each box shape gets its
// own straight-line neighbour arithmetic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "plan.cuh"

namespace cans {
namespace {

struct BoxG {
  int n[3];
  double dxi, dyi, lid;
  const double* dzf;
  const double* dzfi;
  const double* dzci;  // 1 / (centre distance k to k+1), top: the wall ghost (walled) or the wrap (periodic)
  __device__ __forceinline__ size_t at(int i, int j, int k) const {
    return (size_t)i + (size_t)n[0] * ((size_t)j + (size_t)n[1] * k);
  }
  __device__ __forceinline__ double dzc_inv_below(int k) const { return (k == 0) ? dzfi[0] : dzci[k - 1]; }
};

// component C (0 u, 1 v, 2 w) of face field a at (i, j, k), each index at most one cell outside
template <int C, int WX, int WY, int WZ>
__device__ __forceinline__ double V(const BoxG& g, const double* __restrict__ a, int i, int j, int k) {
  const int wl[3] = {WX, WY, WZ};
  int id[3] = {i, j, k};
  double sgn = 1.0, add = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    int& x = id[d];
    if (wl[d] && d == C && (x < 0 || x >= g.n[d] - 1)) return 0.0;
    if (x >= 0 && x < g.n[d]) continue;
    if (!wl[d]) {
      x = (x < 0) ? x + g.n[d] : x - g.n[d];
      continue;
    }
    const bool high = x >= g.n[d];
    x = high ? g.n[d] - 1 : 0;
    add = -add + ((high && d == 2 && C == 0) ? 2.0 * g.lid : 0.0);
    sgn = -sgn;
  }
  return fma(sgn, a[g.at(id[0], id[1], id[2])], add);
}

// cell field with Neumann walls
template <int WX, int WY, int WZ>
__device__ __forceinline__ double Pc(const BoxG& g, const double* __restrict__ q, int i, int j, int k) {
  const int wl[3] = {WX, WY, WZ};
  int id[3] = {i, j, k};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    int& x = id[d];
    if (x >= 0 && x < g.n[d]) continue;
    x = wl[d] ? (x < 0 ? 0 : g.n[d] - 1) : (x < 0 ? x + g.n[d] : x - g.n[d]);
  }
  return q[g.at(id[0], id[1], id[2])];
}

template <int C, int WX, int WY, int WZ>
__device__ __forceinline__ bool wall_face(const BoxG& g, int i, int j, int k) {
  const int wl[3] = {WX, WY, WZ};
  const int x = (C == 0) ? i : (C == 1 ? j : k);
  return wl[C] && x == g.n[C] - 1;
}

// Neighbour access policies: Gen applies every wall and wrap rule; Fast reads at fixed offsets from
// the cell (i0, j0, k0), valid when every neighbour used lies inside the arrays and off the last
// index of each direction (1 <= i <= n - 3 and likewise: then no wrap, no ghost and no wall face
// is touched).
template <int WX, int WY, int WZ>
struct Gen {
  const BoxG& g;
  template <int C>
  __device__ __forceinline__ double vel(const double* a, int i, int j, int k) const {
    return V<C, WX, WY, WZ>(g, a, i, j, k);
  }
  __device__ __forceinline__ double cell(const double* q, int i, int j, int k) const {
    return Pc<WX, WY, WZ>(g, q, i, j, k);
  }
};
struct Fast {
  const BoxG& g;
  int i0, j0, k0;
  size_t c0;
  __device__ __forceinline__ size_t at(int i, int j, int k) const {
    return c0 + (ptrdiff_t)(i - i0) + (ptrdiff_t)(j - j0) * g.n[0] + (ptrdiff_t)(k - k0) * ((ptrdiff_t)g.n[0] * g.n[1]);
  }
  template <int C>
  __device__ __forceinline__ double vel(const double* a, int i, int j, int k) const {
    return a[at(i, j, k)];
  }
  __device__ __forceinline__ double cell(const double* q, int i, int j, int k) const { return q[at(i, j, k)]; }
};
__device__ __forceinline__ bool interior(const BoxG& g, int i, int j, int k) {
  return i >= 1 && i <= g.n[0] - 3 && j >= 1 && j <= g.n[1] - 3 && k >= 1 && k <= g.n[2] - 3;
}

// advection -div(u u) (two-point averages) + nu L at the faces of component C
template <int C, int WX, int WY, int WZ, typename Acc>
__device__ __forceinline__ double box_rhs(const BoxG& g, const Acc& X, const double* u, const double* v,
                                          const double* w, double nu, int i, int j, int k) {
  if (wall_face<C, WX, WY, WZ>(g, i, j, k)) return 0.0;
  auto U = [&](int a, int b, int e) { return X.template vel<0>(u, a, b, e); };
  auto Vv = [&](int a, int b, int e) { return X.template vel<1>(v, a, b, e); };
  auto Ww = [&](int a, int b, int e) { return X.template vel<2>(w, a, b, e); };
  const double* F = (C == 0) ? u : (C == 1 ? v : w);
  auto A = [&](int a, int b, int e) { return X.template vel<C>(F, a, b, e); };
  double adv;
  if (C == 0) {
    const double ue = 0.5 * (U(i, j, k) + U(i + 1, j, k)), uw = 0.5 * (U(i - 1, j, k) + U(i, j, k));
    const double un = 0.25 * (U(i, j, k) + U(i, j + 1, k)) * (Vv(i, j, k) + Vv(i + 1, j, k));
    const double us = 0.25 * (U(i, j - 1, k) + U(i, j, k)) * (Vv(i, j - 1, k) + Vv(i + 1, j - 1, k));
    const double ut = 0.25 * (U(i, j, k) + U(i, j, k + 1)) * (Ww(i, j, k) + Ww(i + 1, j, k));
    const double ub = 0.25 * (U(i, j, k - 1) + U(i, j, k)) * (Ww(i, j, k - 1) + Ww(i + 1, j, k - 1));
    adv = (ue * ue - uw * uw) * g.dxi + (un - us) * g.dyi + (ut - ub) * g.dzfi[k];
  } else if (C == 1) {
    const double ve = 0.25 * (Vv(i, j, k) + Vv(i + 1, j, k)) * (U(i, j, k) + U(i, j + 1, k));
    const double vw = 0.25 * (Vv(i - 1, j, k) + Vv(i, j, k)) * (U(i - 1, j, k) + U(i - 1, j + 1, k));
    const double vn = 0.5 * (Vv(i, j, k) + Vv(i, j + 1, k)), vs = 0.5 * (Vv(i, j - 1, k) + Vv(i, j, k));
    const double vt = 0.25 * (Vv(i, j, k) + Vv(i, j, k + 1)) * (Ww(i, j, k) + Ww(i, j + 1, k));
    const double vb = 0.25 * (Vv(i, j, k - 1) + Vv(i, j, k)) * (Ww(i, j, k - 1) + Ww(i, j + 1, k - 1));
    adv = (ve - vw) * g.dxi + (vn * vn - vs * vs) * g.dyi + (vt - vb) * g.dzfi[k];
  } else {
    const double we = 0.25 * (Ww(i, j, k) + Ww(i + 1, j, k)) * (U(i, j, k) + U(i, j, k + 1));
    const double ww = 0.25 * (Ww(i - 1, j, k) + Ww(i, j, k)) * (U(i - 1, j, k) + U(i - 1, j, k + 1));
    const double wn = 0.25 * (Ww(i, j, k) + Ww(i, j + 1, k)) * (Vv(i, j, k) + Vv(i, j, k + 1));
    const double ws = 0.25 * (Ww(i, j - 1, k) + Ww(i, j, k)) * (Vv(i, j - 1, k) + Vv(i, j - 1, k + 1));
    const double wt = 0.5 * (Ww(i, j, k) + Ww(i, j, k + 1)), wb = 0.5 * (Ww(i, j, k - 1) + Ww(i, j, k));
    adv = (we - ww) * g.dxi + (wn - ws) * g.dyi + (wt * wt - wb * wb) * g.dzci[k];
  }
  const double ac = A(i, j, k);
  const double lx = (A(i - 1, j, k) - 2 * ac + A(i + 1, j, k)) * g.dxi * g.dxi;
  const double ly = (A(i, j - 1, k) - 2 * ac + A(i, j + 1, k)) * g.dyi * g.dyi;
  double lz;
  if (C < 2) {
    lz = ((A(i, j, k + 1) - ac) * g.dzci[k] - (ac - A(i, j, k - 1)) * g.dzc_inv_below(k)) * g.dzfi[k];
  } else {
    const int ku = (k + 1 < g.n[2]) ? k + 1 : 0;
    lz = ((A(i, j, k + 1) - ac) * g.dzfi[ku] - (ac - A(i, j, k - 1)) * g.dzfi[k]) * g.dzci[k];
  }
  return fma(nu, lx + ly + lz, -adv);
}

template <int C, int WX, int WY, int WZ, typename Acc>
__device__ __forceinline__ double grad(const BoxG& g, const Acc& X, const double* q, int i, int j, int k) {
  if (wall_face<C, WX, WY, WZ>(g, i, j, k)) return 0.0;
  const double qc = q[g.at(i, j, k)];
  if (C == 0) return (X.cell(q, i + 1, j, k) - qc) * g.dxi;
  if (C == 1) return (X.cell(q, i, j + 1, k) - qc) * g.dyi;
  return (X.cell(q, i, j, k + 1) - qc) * g.dzci[k];
}

template <int WX, int WY, int WZ>
__global__ void box_momentum_kernel(BoxG g, const double* __restrict__ u, const double* __restrict__ v,
                                    const double* __restrict__ w, const double* __restrict__ p, double* __restrict__ ru,
                                    double* __restrict__ rv, double* __restrict__ rw, double* __restrict__ us,
                                    double* __restrict__ vs, double* __restrict__ ws, double nu, double alpha,
                                    double beta, double gamma, const double* __restrict__ dt_dev) {
  const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
  const double dt = *dt_dev;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % g.n[0]), j = (int)((c / g.n[0]) % g.n[1]), k = (int)(c / ((size_t)g.n[0] * g.n[1]));
    auto body = [&](const auto& X) {
      const double r0 = box_rhs<0, WX, WY, WZ>(g, X, u, v, w, nu, i, j, k);
      const double r1 = box_rhs<1, WX, WY, WZ>(g, X, u, v, w, nu, i, j, k);
      const double r2 = box_rhs<2, WX, WY, WZ>(g, X, u, v, w, nu, i, j, k);
      double s0 = alpha * r0, s1 = alpha * r1, s2 = alpha * r2;
      if (beta != 0.0) {
        s0 = fma(beta, ru[c], s0);
        s1 = fma(beta, rv[c], s1);
        s2 = fma(beta, rw[c], s2);
      }
      us[c] = fma(dt, fma(-gamma, grad<0, WX, WY, WZ>(g, X, p, i, j, k), s0), u[c]);
      vs[c] = fma(dt, fma(-gamma, grad<1, WX, WY, WZ>(g, X, p, i, j, k), s1), v[c]);
      ws[c] = fma(dt, fma(-gamma, grad<2, WX, WY, WZ>(g, X, p, i, j, k), s2), w[c]);
      ru[c] = r0;
      rv[c] = r1;
      rw[c] = r2;
    };
    if (interior(g, i, j, k))
      body(Fast{g, i, j, k, c});
    else
      body(Gen<WX, WY, WZ>{g});
  }
}

template <int WX, int WY, int WZ>
__global__ void box_divergence_kernel(BoxG g, const double* __restrict__ u, const double* __restrict__ v,
                                      const double* __restrict__ w, double* __restrict__ f, double gamma,
                                      const double* __restrict__ dt_dev) {
  const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
  const double scale = 1.0 / (gamma * (*dt_dev));
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % g.n[0]), j = (int)((c / g.n[0]) % g.n[1]), k = (int)(c / ((size_t)g.n[0] * g.n[1]));
    auto div = [&](const auto& X) {
      return (X.template vel<0>(u, i, j, k) - X.template vel<0>(u, i - 1, j, k)) * g.dxi +
             (X.template vel<1>(v, i, j, k) - X.template vel<1>(v, i, j - 1, k)) * g.dyi +
             (X.template vel<2>(w, i, j, k) - X.template vel<2>(w, i, j, k - 1)) * g.dzfi[k];
    };
    const double d = interior(g, i, j, k) ? div(Fast{g, i, j, k, c}) : div(Gen<WX, WY, WZ>{g});
    f[c] = scale * d;
  }
}

template <int WX, int WY, int WZ>
__global__ void box_correct_kernel(BoxG g, const double* __restrict__ us, const double* __restrict__ vs,
                                   const double* __restrict__ ws, const double* __restrict__ phi,
                                   double* __restrict__ u, double* __restrict__ v, double* __restrict__ w,
                                   double* __restrict__ p, double gamma, const double* __restrict__ dt_dev,
                                   DetSum bulk) {
  const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
  const double f = gamma * (*dt_dev);
  double acc = 0.0;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % g.n[0]), j = (int)((c / g.n[0]) % g.n[1]), k = (int)(c / ((size_t)g.n[0] * g.n[1]));
    double gx, gy, gz;
    auto grads = [&](const auto& X) {
      gx = grad<0, WX, WY, WZ>(g, X, phi, i, j, k);
      gy = grad<1, WX, WY, WZ>(g, X, phi, i, j, k);
      gz = grad<2, WX, WY, WZ>(g, X, phi, i, j, k);
    };
    if (interior(g, i, j, k))
      grads(Fast{g, i, j, k, c});
    else
      grads(Gen<WX, WY, WZ>{g});
    const double un = us[c] - f * gx;
    u[c] = un;
    v[c] = vs[c] - f * gy;
    w[c] = ws[c] - f * gz;
    p[c] += phi[c];
    acc += g.dzf[k] * un;
  }
  if (bulk.out != nullptr) det_sum_finish(block_sum_d(acc), bulk);
}

template <int WX, int WY, int WZ>
__global__ void box_chkdt_kernel(BoxG g, const double* __restrict__ u, const double* __restrict__ v,
                                 const double* __restrict__ w, unsigned long long* dti_bits) {
  const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
  double dti = 0.0;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % g.n[0]), j = (int)((c / g.n[0]) % g.n[1]), k = (int)(c / ((size_t)g.n[0] * g.n[1]));
    auto dti_at = [&](const auto& X) {
    auto U = [&](int a, int b, int e) { return X.template vel<0>(u, a, b, e); };
    auto Vv = [&](int a, int b, int e) { return X.template vel<1>(v, a, b, e); };
    auto Ww = [&](int a, int b, int e) { return X.template vel<2>(w, a, b, e); };
    const double dtix = fabs(U(i, j, k)) * g.dxi +
                        0.25 * fabs(Vv(i, j, k) + Vv(i, j - 1, k) + Vv(i + 1, j, k) + Vv(i + 1, j - 1, k)) * g.dyi +
                        0.25 * fabs(Ww(i, j, k) + Ww(i, j, k - 1) + Ww(i + 1, j, k) + Ww(i + 1, j, k - 1)) * g.dzfi[k];
    const double dtiy = 0.25 * fabs(U(i, j, k) + U(i - 1, j, k) + U(i, j + 1, k) + U(i - 1, j + 1, k)) * g.dxi +
                        fabs(Vv(i, j, k)) * g.dyi +
                        0.25 * fabs(Ww(i, j, k) + Ww(i, j, k - 1) + Ww(i, j + 1, k) + Ww(i, j + 1, k - 1)) * g.dzfi[k];
    const double dtiz = 0.25 * fabs(U(i, j, k) + U(i - 1, j, k) + U(i, j, k + 1) + U(i - 1, j, k + 1)) * g.dxi +
                        0.25 * fabs(Vv(i, j, k) + Vv(i, j - 1, k) + Vv(i, j, k + 1) + Vv(i, j - 1, k + 1)) * g.dyi +
                        fabs(Ww(i, j, k)) * g.dzci[k];
    return fmax(dtix, fmax(dtiy, dtiz));
    };
    dti = fmax(dti, interior(g, i, j, k) ? dti_at(Fast{g, i, j, k, c}) : dti_at(Gen<WX, WY, WZ>{g}));
  }
  for (int o = 16; o > 0; o >>= 1) dti = fmax(dti, __shfl_xor_sync(0xffffffffu, dti, o));
  if ((threadIdx.x & 31) == 0) atomicMax(dti_bits, (unsigned long long)__double_as_longlong(dti));
}

__global__ void box_dt_kernel(const unsigned long long* dti_bits, double* dt_dev, double cfl, double nu, double dl,
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

__global__ void box_forcing_kernel(size_t N, double* __restrict__ u, const double* __restrict__ bulk, double inv_vol,
                                   double ubulk) {
  const double shift = ubulk - (*bulk) * inv_vol;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x)
    u[c] += shift;
}

int grid_for(size_t N) { return (int)std::min<size_t>((N + 255) / 256, (size_t)148 * 16); }

template <int WX, int WY, int WZ>
int box_step(const cans_plan_s* P, double* u, double* v, double* w, double* p, const cans_rk3_params* prm, double lid,
             double* dt, unsigned char* base, size_t fb, void* pws, double* small, cudaStream_t st) {
  const double ALPHA[3] = {8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0};
  const double BETA[3] = {0.0, -17.0 / 60.0, -5.0 / 12.0};
  BoxG g;
  for (int d = 0; d < 3; ++d) g.n[d] = P->n[d];
  g.dxi = P->n[0] / P->len[0];
  g.dyi = P->n[1] / P->len[1];
  g.lid = lid;
  g.dzf = P->dzf_d;
  g.dzfi = P->dzfi_d;
  g.dzci = P->dzci_d;
  const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
  double* F[8];
  for (int q = 0; q < 8; ++q) F[q] = reinterpret_cast<double*>(base + q * fb);
  double *us = F[0], *vs = F[1], *ws = F[2], *ru = F[3], *rv = F[4], *rw = F[5], *f = F[6], *phi = F[7];
  const int G = grid_for(N);
  unsigned long long* dti = reinterpret_cast<unsigned long long*>(small + 2);
#define BOX_CK(...)                                  \
  do {                                               \
    if ((__VA_ARGS__) != cudaSuccess) return CANS_ERR_CUDA; \
  } while (0)
  cans_plan_t PM = const_cast<cans_plan_t>(P);  // the profile records live in the plan
  double dl = std::min(P->len[0] / P->n[0], P->len[1] / P->n[1]);
  for (int k = 0; k < P->n[2]; ++k) dl = std::min(dl, P->dzf_h[k]);
  {
    PassTimer tm(PM, CANS_PASS_CHKDT, st);
    BOX_CK(cudaMemsetAsync(dti, 0, sizeof(unsigned long long), st));
    if (!(prm->dt > 0)) box_chkdt_kernel<WX, WY, WZ><<<G, 256, 0, st>>>(g, u, v, w, dti);
    box_dt_kernel<<<1, 32, 0, st>>>(dti, dt, prm->cfl, prm->nu, dl, prm->dt);
    BOX_CK(cudaGetLastError());
  }
  double lz = 0;
  for (int k = 0; k < P->n[2]; ++k) lz += P->dzf_h[k];
  for (int s = 0; s < 3; ++s) {
    const double a = ALPHA[s], b = BETA[s], gm = a + b;
    {
      PassTimer tm(PM, CANS_PASS_MOMENTUM, st);
      box_momentum_kernel<WX, WY, WZ><<<G, 256, 0, st>>>(g, u, v, w, p, ru, rv, rw, us, vs, ws, prm->nu, a, b, gm, dt);
    }
    {
      PassTimer tm(PM, CANS_PASS_DIVERGENCE, st);
      box_divergence_kernel<WX, WY, WZ><<<G, 256, 0, st>>>(g, us, vs, ws, f, gm, dt);
    }
    BOX_CK(cudaGetLastError());
    const int rc = cans_poisson_solve(PM, f, phi, pws, st, nullptr);
    if (rc != CANS_OK) return rc;
    double* bulk = prm->forcing ? small + 1 : nullptr;
    {
      PassTimer tm(PM, CANS_PASS_CORRECT, st);
      if ((size_t)G > PM->dsum_nslots) return CANS_ERR_CUDA;
      box_correct_kernel<WX, WY, WZ><<<G, 256, 0, st>>>(g, us, vs, ws, phi, u, v, w, p, gm, dt, plan_sum(PM, bulk));
    }
    if (bulk) {
      PassTimer tm(PM, CANS_PASS_FORCING, st);
      box_forcing_kernel<<<G, 256, 0, st>>>(N, u, bulk, 1.0 / ((double)g.n[0] * g.n[1] * lz), prm->ubulk);
    }
    BOX_CK(cudaGetLastError());
  }
#undef BOX_CK
  return CANS_OK;
}

size_t a256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace
}  // namespace cans

using namespace cans;

extern "C" {

int cans_box_rk3_workspace_size(cans_plan_t P, size_t* bytes) {
  if (!P || !bytes) return CANS_ERR_ARG;
  const size_t N = (size_t)P->n[0] * P->n[1] * P->n[2];
  size_t pws = 0;
  cans_poisson_workspace_size(P, &pws);
  *bytes = 8 * a256(N * sizeof(double)) + 256 + a256(pws);
  return CANS_OK;
}

int cans_box_rk3_step(cans_plan_t P, double* u, double* v, double* w, double* p, const cans_rk3_params* prm,
                      double lid, double* dt_dev, void* workspace, void* cuda_stream) {
  if (!P || !u || !v || !w || !p || !prm || !workspace) return CANS_ERR_ARG;
  for (int d = 0; d < 3; ++d)
    if (P->bc[d] != BC_P && P->bc[d] != BC_NN) return CANS_ERR_UNSUPPORTED;
  if (P->opts.z_grid != 0 || P->opts.shift != 0.0) return CANS_ERR_UNSUPPORTED;
  if (!(prm->nu > 0) || !(prm->cfl > 0) || !std::isfinite(lid)) return CANS_ERR_ARG;
  if (lid != 0.0 && P->bc[2] != BC_NN) return CANS_ERR_ARG;  // the lid is the top z wall
  for (int d = 0; d < 3; ++d)
    if (P->bc[d] == BC_NN && P->n[d] < 2) return CANS_ERR_UNSUPPORTED;  // a walled direction needs a face inside
  if (reinterpret_cast<uintptr_t>(workspace) & 255) return CANS_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const size_t N = (size_t)P->n[0] * P->n[1] * P->n[2];
  const size_t fb = a256(N * sizeof(double));
  unsigned char* base = static_cast<unsigned char*>(workspace);
  double* small = reinterpret_cast<double*>(base + 8 * fb);  // [0] dt, [1] bulk sum, [2] dti bits
  void* pws = base + 8 * fb + 256;
  double* dt = dt_dev ? dt_dev : small;
  const int wx = P->bc[0] == BC_NN, wy = P->bc[1] == BC_NN, wz = P->bc[2] == BC_NN;
  switch (wx * 4 + wy * 2 + wz) {
    case 0: return box_step<0, 0, 0>(P, u, v, w, p, prm, lid, dt, base, fb, pws, small, st);
    case 1: return box_step<0, 0, 1>(P, u, v, w, p, prm, lid, dt, base, fb, pws, small, st);
    case 2: return box_step<0, 1, 0>(P, u, v, w, p, prm, lid, dt, base, fb, pws, small, st);
    case 3: return box_step<0, 1, 1>(P, u, v, w, p, prm, lid, dt, base, fb, pws, small, st);
    case 4: return box_step<1, 0, 0>(P, u, v, w, p, prm, lid, dt, base, fb, pws, small, st);
    case 5: return box_step<1, 0, 1>(P, u, v, w, p, prm, lid, dt, base, fb, pws, small, st);
    case 6: return box_step<1, 1, 0>(P, u, v, w, p, prm, lid, dt, base, fb, pws, small, st);
    default: return box_step<1, 1, 1>(P, u, v, w, p, prm, lid, dt, base, fb, pws, small, st);
  }
}

}  // extern "C"
