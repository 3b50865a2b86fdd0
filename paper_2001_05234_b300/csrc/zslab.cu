// The z solve of one Poisson problem split over P ranks by z-slabs (the paper's Implementation section
// distributes the grid over GPUs; here the x-y transforms stay local to a rank's slab and only the
// tridiagonal systems of Eq. poi_reduced cross the slab boundaries).
//
// Rank r owns rows z0 .. z1-1 of every column's system.  The elimination pass runs Thomas' forward
// sweep over the slab with two extra right-hand sides (the couplings to L_{r-1}, the last unknown of the
// previous slab, and to L_r, the slab's own last unknown), so that each interior row reads
//   x_k = D_k + V_k L_{r-1} + W_k L_r,
// and it publishes, per column, the expressions of the slab's first and last interior rows and the
// coefficients of its last row (10 numbers).  With every rank's numbers gathered, the last rows give
// one tridiagonal system of P unknowns per column -- the same reduced system the warp-level
// partitioned solve of the single-GPU z pass forms across lanes -- which every rank solves; the finish
// pass then back-substitutes its slab.  The singular (0,0) mode of a problem without Dirichlet
// directions is solved whole on every rank from its gathered right-hand side (Nz numbers), with the
// compatible projection and zero weighted mean of the single-GPU solve.  All in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <vector>

#include "plan.cuh"

struct cans_zslab_s {
  cans_plan_t plan;  // the whole problem's plan (its z rows, eigenvalues and dzf)
  int z0, z1, nzs;   // this rank's rows
  double* tab = nullptr;  // device: the slab's rows a, b, c (3 nzs)
};

namespace cans {
namespace {

constexpr int kIface = 10;  // Df, Vf, Wf (first row), Dl, Vl, Wl (last interior row), al, bl, cl, dl (last row)

// One thread per (i, j) column: the slab's forward sweep with the two coupling columns; the modified
// right-hand side dp overwrites the field in place, the pivots' c' and the L_{r-1} column l' go to the
// workspace (2 nzs doubles per column), the back sweep of the expressions gives D, V, W of the first
// and the last interior row.
__global__ void zslab_eliminate_kernel(double* __restrict__ x, double* __restrict__ cw, double* __restrict__ lw,
                                       double* __restrict__ iface, double* __restrict__ col00, const double* a,
                                       const double* b, const double* c, const double* mux, const double* muy,
                                       double shift, int nx, int ny, int nzs, int singular) {
  const size_t ncol = (size_t)nx * ny;
  const size_t col = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (col >= ncol) return;
  const int i = (int)(col % nx), j = (int)(col / nx);
  const double mu = mux[i] + muy[j] + shift;
  if (singular && col == 0) {  // the singular mode is solved whole in the finish pass
    for (int r = 0; r < nzs; ++r) col00[r] = x[(size_t)r * ncol];
  }
  double* out = iface + col * kIface;
  double cprev = 0, dprev = 0, lprev = 0;
  // rows 0 .. nzs-2 eliminated; row nzs-1 (the slab's last row, unknown L_r) stays
  for (int r = 0; r + 1 < nzs; ++r) {
    const size_t o = (size_t)r * ncol + col;
    const double ar = a[r], br = b[r] + mu, cr = c[r];
    const double inv = 1.0 / (br - ar * cprev);
    const bool last_inner = (r == nzs - 2);
    const double cp = last_inner ? 0.0 : cr * inv;  // the last interior row couples to L_r instead
    const double dp = (x[o] - ar * dprev) * inv;
    const double lp = ((r == 0) ? -ar : -ar * lprev) * inv;
    x[o] = dp;
    cw[o] = last_inner ? -cr * inv : cp;  // the last interior row keeps its coupling -c/pivot to L_r
    lw[o] = lp;
    cprev = cp;
    dprev = dp;
    lprev = lp;
  }
  // back sweep of the expressions x_r = D + V L_{r-1} + W L_r
  double Df = 0, Vf = 0, Wf = 1, Dl = 0, Vl = 1, Wl = 0;
  if (nzs >= 2) {
    double D = 0, V = 0, W = 0;
    for (int r = nzs - 2; r >= 0; --r) {
      const size_t o = (size_t)r * ncol + col;
      if (r == nzs - 2) {
        D = x[o];
        V = lw[o];
        W = cw[o];
        Dl = D;
        Vl = V;
        Wl = W;
      } else {
        D = x[o] - cw[o] * D;
        V = lw[o] - cw[o] * V;
        W = -cw[o] * W;
      }
    }
    Df = D;
    Vf = V;
    Wf = W;
  }
  const int rl = nzs - 1;
  out[0] = Df;
  out[1] = Vf;
  out[2] = Wf;
  out[3] = Dl;
  out[4] = Vl;
  out[5] = Wl;
  out[6] = a[rl];
  out[7] = b[rl] + mu;
  out[8] = c[rl];
  out[9] = x[(size_t)rl * ncol + col];
}

// One thread per column: the reduced system of the P slabs' last rows (Thomas, P unknowns), then this
// rank's back substitution x_r = D_r + V_r L_{rank-1} + W_r L_rank over its interior rows, x = L_rank on
// its last row, everything times `scale`.  iface_all: P blocks of ncol x kIface, rank-major.
__global__ void zslab_finish_kernel(double* __restrict__ x, const double* __restrict__ cw,
                                    const double* __restrict__ lw, const double* __restrict__ iface_all, int nranks,
                                    int rank, int nx, int ny, int nzs, double scale, int skip00) {
  const size_t ncol = (size_t)nx * ny;
  const size_t col = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (col >= ncol || (skip00 && col == 0)) return;
  constexpr int PMAX = 64;
  double cs[PMAX], ds[PMAX];
  auto F = [&](int q, int e) { return iface_all[((size_t)q * ncol + col) * kIface + e]; };
  // equation q: alpha_q L_{q-1} + beta_q L_q + gamma_q L_{q+1} = delta_q
  double cprev = 0, dprev = 0;
  for (int q = 0; q < nranks; ++q) {
    const double al = F(q, 6), bl = F(q, 7), cl = F(q, 8), dl = F(q, 9);
    const double Dl = F(q, 3), Vl = F(q, 4), Wl = F(q, 5);
    const bool hasn = q + 1 < nranks;
    const double Dfn = hasn ? F(q + 1, 0) : 0.0, Vfn = hasn ? F(q + 1, 1) : 0.0, Wfn = hasn ? F(q + 1, 2) : 0.0;
    const double alpha = (q == 0) ? 0.0 : al * Vl;
    const double beta = bl + al * Wl + (hasn ? cl * Vfn : 0.0);
    const double gamma = hasn ? cl * Wfn : 0.0;
    const double delta = dl - al * Dl - (hasn ? cl * Dfn : 0.0);
    const double inv = 1.0 / (beta - alpha * cprev);
    cs[q] = gamma * inv;
    ds[q] = (delta - alpha * dprev) * inv;
    cprev = cs[q];
    dprev = ds[q];
  }
  double Lq = ds[nranks - 1], Lown = 0.0, Lprev = 0.0;
  for (int q = nranks - 1; q >= 0; --q) {
    if (q < nranks - 1) Lq = ds[q] - cs[q] * Lq;
    if (q == rank) Lown = Lq;
    if (q == rank - 1) Lprev = Lq;
  }
  // back substitution of the slab: x_{nzs-1} = L_own, x_r = dp_r + l'_r L_prev - c'_r x_{r+1}
  double xn = Lown;
  x[(size_t)(nzs - 1) * ncol + col] = scale * Lown;
  for (int r = nzs - 2; r >= 0; --r) {
    const size_t o = (size_t)r * ncol + col;
    xn = (r == nzs - 2) ? x[o] + lw[o] * Lprev + cw[o] * Lown : x[o] + lw[o] * Lprev - cw[o] * xn;
    x[o] = scale * xn;
  }
}

// The singular (0,0) column solved whole (one thread): the gathered right-hand side d (Nz), the
// compatible projection sum_k dzf_k d_k = 0, the last row replaced by x = 0, Thomas, the zero
// dzf-weighted mean; this rank's rows z0 .. z0+nzs-1 written to the field, times `scale`.
__global__ void zslab_col00_kernel(double* __restrict__ x, double* __restrict__ d, const double* a, const double* b,
                                   const double* c, const double* dzf, int nz, int z0, int nzs, size_t ncol,
                                   double scale, double* __restrict__ cwork) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double sw = 0, swd = 0;
  for (int k = 0; k < nz; ++k) {
    sw += dzf[k];
    swd += dzf[k] * d[k];
  }
  const double proj = swd / sw;
  double cprev = 0, dprev = 0;
  for (int k = 0; k < nz; ++k) {
    double ak = a[k], bk = b[k], ck = c[k], dk = d[k] - proj;
    if (k == nz - 1) {
      ak = 0;
      bk = 1;
      ck = 0;
      dk = 0;
    }
    const double inv = 1.0 / (bk - ak * cprev);
    cwork[k] = ck * inv;
    d[k] = (dk - ak * dprev) * inv;
    cprev = cwork[k];
    dprev = d[k];
  }
  for (int k = nz - 2; k >= 0; --k) d[k] -= cwork[k] * d[k + 1];
  double sx = 0;
  for (int k = 0; k < nz; ++k) sx += dzf[k] * d[k];
  const double mean = sx / sw;
  for (int r = 0; r < nzs; ++r) x[(size_t)r * ncol] = scale * (d[z0 + r] - mean);
}

}  // namespace
}  // namespace cans

using namespace cans;

extern "C" {

int cans_zslab_create(cans_plan_t P, int z0, int z1, cans_zslab_t* out) {
  if (!P || !out) return CANS_ERR_ARG;
  *out = nullptr;
  if (P->opts.prec != CANS_FP64 || P->bc[2] == BC_P || P->opts.z_grid != 0) return CANS_ERR_UNSUPPORTED;
  if (z0 < 0 || z1 <= z0 || z1 > P->n[2]) return CANS_ERR_ARG;
  cans_zslab_s* S = new (std::nothrow) cans_zslab_s();
  if (!S) return CANS_ERR_ARG;
  S->plan = P;
  S->z0 = z0;
  S->z1 = z1;
  S->nzs = z1 - z0;
  // the whole problem's z rows (wall rows included), this slab's part
  const int nz = P->n[2];
  std::vector<double> ha(nz), hb(nz), hc(nz);
  if (cudaMemcpy(ha.data(), P->zt_d.a, nz * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(hb.data(), P->zt_d.b, nz * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(hc.data(), P->zt_d.c, nz * 8, cudaMemcpyDeviceToHost) != cudaSuccess) {
    delete S;
    return CANS_ERR_CUDA;
  }
  std::vector<double> t(3 * (size_t)S->nzs);
  for (int r = 0; r < S->nzs; ++r) {
    t[r] = ha[z0 + r];
    t[S->nzs + r] = hb[z0 + r];
    t[2 * S->nzs + r] = hc[z0 + r];
  }
  if (cudaMalloc(&S->tab, t.size() * 8) != cudaSuccess ||
      cudaMemcpy(S->tab, t.data(), t.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
    if (S->tab) cudaFree(S->tab);
    delete S;
    return CANS_ERR_CUDA;
  }
  *out = S;
  return CANS_OK;
}

int cans_zslab_sizes(cans_zslab_t S, size_t* workspace_bytes, size_t* iface_doubles, size_t* col00_doubles) {
  if (!S) return CANS_ERR_ARG;
  const size_t ncol = (size_t)S->plan->n[0] * S->plan->n[1];
  if (workspace_bytes) *workspace_bytes = 2 * ncol * S->nzs * sizeof(double) + 2 * (size_t)S->plan->n[2] * 8 + 256;
  if (iface_doubles) *iface_doubles = ncol * kIface;
  if (col00_doubles) *col00_doubles = (size_t)S->nzs;
  return CANS_OK;
}

int cans_zslab_eliminate(cans_zslab_t S, double* field, double* iface, double* col00, void* workspace,
                         void* cuda_stream) {
  if (!S || !field || !iface || !col00 || !workspace) return CANS_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(workspace) & 255) return CANS_ERR_WORKSPACE;
  const cans_plan_s* P = S->plan;
  const size_t ncol = (size_t)P->n[0] * P->n[1];
  double* cw = static_cast<double*>(workspace);
  double* lw = cw + ncol * S->nzs;
  const int blocks = (int)((ncol + 255) / 256);
  zslab_eliminate_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
      field, cw, lw, iface, col00, S->tab, S->tab + S->nzs, S->tab + 2 * S->nzs, P->mux_d, P->muy_d, P->shift,
      P->n[0], P->n[1], S->nzs, P->singular ? 1 : 0);
  return cudaGetLastError() == cudaSuccess ? CANS_OK : CANS_ERR_CUDA;
}

int cans_zslab_finish(cans_zslab_t S, double* field, const double* iface_all, const double* col00_all, int nranks,
                      int rank, double scale, void* workspace, void* cuda_stream) {
  if (!S || !field || !iface_all || !workspace || nranks < 1 || nranks > 64 || rank < 0 || rank >= nranks)
    return CANS_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(workspace) & 255) return CANS_ERR_WORKSPACE;
  const cans_plan_s* P = S->plan;
  if (P->singular && !col00_all) return CANS_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const size_t ncol = (size_t)P->n[0] * P->n[1];
  double* cw = static_cast<double*>(workspace);
  double* lw = cw + ncol * S->nzs;
  const int blocks = (int)((ncol + 255) / 256);
  zslab_finish_kernel<<<blocks, 256, 0, st>>>(field, cw, lw, iface_all, nranks, rank, P->n[0], P->n[1], S->nzs, scale,
                                              P->singular ? 1 : 0);
  if (cudaGetLastError() != cudaSuccess) return CANS_ERR_CUDA;
  if (P->singular) {
    // the gathered (0,0) column is copied to the workspace's tail, solved whole there
    double* d = lw + ncol * S->nzs;
    double* cwork = d + P->n[2];
    if (cudaMemcpyAsync(d, col00_all, P->n[2] * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return CANS_ERR_CUDA;
    zslab_col00_kernel<<<1, 32, 0, st>>>(field, d, P->zt_d.a, P->zt_d.b, P->zt_d.c, P->dzf_d, P->n[2], S->z0, S->nzs,
                                         ncol, scale, cwork);
    if (cudaGetLastError() != cudaSuccess) return CANS_ERR_CUDA;
  }
  return CANS_OK;
}

int cans_zslab_destroy(cans_zslab_t S) {
  if (!S) return CANS_ERR_ARG;
  if (S->tab) cudaFree(S->tab);
  delete S;
  return CANS_OK;
}

}  // extern "C"
