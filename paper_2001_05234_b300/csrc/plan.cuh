// Plan object shared by the host code and the pass launchers (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "cans.h"
#include "detsum.cuh"
#include "dfloat.cuh"
#include "lines.cuh"
#include "zsolve.cuh"

namespace cans {

struct DirHost {
  int n = 1, m = 0, bc = 0, nst = 0;
  int radix[16] = {0};
};

struct Launch {
  int nl = 1, lognl = 0, threads = 32;
  size_t smem = 0;
};

// Stencil coefficients for the residual r = f - L_h p (Eq. poi with a non-uniform z).
struct StencilDF {
  df idx2, idy2;
  df shift;  // Helmholtz shift sigma of (L_h + sigma): 0 for Poisson
  const float *sa_hi, *sa_lo, *sc_hi, *sc_lo;  // z: a_k (to k-1), c_k (to k+1), wall ghosts included
  int bc[3];
  int xlo, xhi, ylo, yhi, zlo, zhi;  // wall rule (BC_NN or BC_DD) at the low and the high wall of each walled direction
  int n[3];
  int iso;  // 1/dx^2 == 1/dy^2 exactly
};

// Layout of a transformed work field.  natural: [k][j][i] (x fastest, as the user's fields);
// blocked: [k][i / 32][j][i % 32] -- 32 consecutive x-slots of every (j, k) stay together, so a y-pass
// tile of up to 32 x-slots reads consecutive 128-byte rows and a z-pass tile reads 128-byte rows.
struct WLay {
  int blk, nx, ny, nbx;  // nbx = number of 32-slot blocks per line (blocked layout)
  __device__ __forceinline__ size_t at(int i, int j, int k) const {
    if (!blk) return (size_t)i + (size_t)nx * ((size_t)j + (size_t)ny * k);
    return ((size_t)k * nbx + (i >> 5)) * ((size_t)ny * 32) + (size_t)j * 32 + (i & 31);
  }
  // y-pass tile of x-slots i0 .. (i0 + nl - 1 within one block) at plane k: element (l, j) = base + j*rs + l
  __device__ __forceinline__ size_t ybase(int i0, int k) const { return at(i0, 0, k); }
  __device__ __forceinline__ int yrow() const { return blk ? 32 : nx; }
  // z-pass tile of x-slots i0.. at y-slot j: element (ii, k) = base + k*zs + ii
  __device__ __forceinline__ size_t zbase(int i0, int j) const { return at(i0, j, 0); }
  __device__ __forceinline__ size_t zstride() const { return blk ? (size_t)nbx * ny * 32 : (size_t)nx * ny; }
};

// The right-hand side of Eq. poi_ns formed from the face velocities of a channel (x, y periodic, w = 0
// on both wall faces): f = s (dxi (u_i - u_{i-1}) + dyi (v_j - v_{j-1}) + dzfi_k (w_k - w_{k-1})) with
// s = num / (gamma dt), dt read on the device (s = num when dt is NULL).  The fused multiply-adds are
// spelled out, so the stand-alone divergence kernel and the x pass that forms f on the fly produce the
// same bits (and the FP64 operation count stays at seven per point).
struct DivArgs {
  const double *u, *v, *w;
  double* fout;  // optional: f written as a by-product (the mixed refinement's residual reads it)
  const double* dzfi;
  const double* dt;
  double num, gamma, dxi, dyi;
  int nx, ny, nz;
  __device__ __forceinline__ double scale() const { return dt != nullptr ? num / (gamma * (*dt)) : num; }
  // f at cell (i, j, k), linear index c
  __device__ __forceinline__ double at(double s, size_t c, int i, int j, int k) const {
    const size_t im = (i == 0) ? c + (size_t)(nx - 1) : c - 1;
    const size_t jm = (j == 0) ? c + (size_t)(ny - 1) * nx : c - (size_t)nx;
    const double wt = (k < nz - 1) ? w[c] : 0.0;
    const double wb = (k >= 1) ? w[c - (size_t)nx * ny] : 0.0;
    const double t = __fma_rn(__dsub_rn(u[c], u[im]), dxi,
                              __fma_rn(__dsub_rn(v[c], v[jm]), dyi, __dmul_rn(__dsub_rn(wt, wb), dzfi[k])));
    return __dmul_rn(s, t);
  }
};

struct XArgs {
  int nx, nlines, lognl;
  double scale;  // inverse only
  WLay w;        // layout of the transformed field (xfwd output, xinv input)
};

struct ZArgs {
  int nx, ny, nz, ti, m;
  int singular;               // the (0,0) mode is singular (Neumann z, no Dirichlet direction, no shift)
  double shift;               // Helmholtz shift added to every diagonal (0 for Poisson)
  const unsigned char* mask;  // mixed: 1 = solve this column in double
  const double* mux_d;
  const double* muy_d;
  const float* mux_f;
  const float* muy_f;
  const double* dzf;
  const double* gauge;  // optional: target weighted column mean = gauge_scale * (*gauge)
  double gauge_scale;
  int j_end, i_end;     // FP64-column kernel: bounding box of the columns it owns
  int xpairs;           // x periodic, even widths: column pairs of equal shift
  double* compat;       // optional: sum_k dzf_k d_k of the singular column (before its projection)
  int* status;          // plan status word (bounded waits record CANS_ERR_TIMEOUT here)
};

}  // namespace cans

struct cans_plan_s {
  int n[3];
  double len[2];
  int bc[3];
  cans_opts opts;
  int device = 0;
  bool sing_bc = false;   // no Dirichlet direction: singular unless shifted
  bool singular = false;  // sing_bc and a zero shift for the solve in progress
  double shift = 0;       // Helmholtz shift of the solve in progress (opts.shift by default)
  int nz_cells = 0;       // cells of the caller's dzf (n[2] + 1 on the face grid)
  cans::DirHost dx, dy, dz;  // dz only for a periodic z
  std::vector<double> mux_h, muy_h;
  void* dtab = nullptr;
  cans::LineTab<double> tx_d, ty_d;
  cans::LineTab<float> tx_f, ty_f;
  cans::LineTab<double> tz_d;  // periodic z only
  cans::LineTab<float> tz_f;
  const double* muz_d = nullptr;
  const float* muz_f = nullptr;
  cans::Launch zs_l[2];
  cans::ZTab<double> zt_d;
  cans::ZTab<float> zt_f;
  const double *mux_d, *muy_d, *dzf_d, *sa_d, *sc_d;
  const float* dzf_f;
  const float* dzf_flo;  // dzf - (float)dzf
  const double* dzfi_d;  // 1/dzf
  const double* dzci_d;  // 1/dzc_{k+1/2} (top: 1/dzf of the wall cell)
  std::vector<double> dzf_h;
  double gauge_scale = 0;
  const float *mux_f, *muy_f, *sa_hi, *sa_lo, *sc_hi, *sc_lo;
  const unsigned char* mask_d = nullptr;
  int mask_i_end = 0, mask_j_end = 0;  // bounding box of the double-precision columns (mixed)
  double* acc_d = nullptr;             // [0] |f|^2, [1+s] |r_s|^2, [nacc-7] compatibility sum,
                                       // [nacc-5] gauge sum, [nacc-4..] reports
  int nacc = 0;
  int* status_d = nullptr;             // device status word (cans_plan_status)
  double* dsum_slots = nullptr;        // per-block slots of the reproducible sums (detsum.cuh) ...
  unsigned* dsum_count = nullptr;      // ... and their arrival counter
  size_t dsum_nslots = 0;              // slots: one per x line, at least 148 * 16 (every grid that sums)
  double compat_scale = 0;             // sqrt(Nx Ny sum_k dzf_k^2): |sum w f| <= compat_scale ||f||_2
  double idx2, idy2;
  cans::Launch x_l[2], y_l[2];  // [0] double storage, [1] float storage
  int z_ti[2], z_m, z_mmax;
  int res_split = 1;  // CTA-engine x lines: the sweep residual as the streaming stencil + an x pass from
                      // 2^24 points on (1), never (0), always (2); fused into the x pass otherwise
  int res_pts = 4;  // residual stencil: points per thread (4, 2 or 1; fewer where nx or alignment demand)
  int z_fuse64 = 1;  // staged float z kernel, <= 4 rows per lane: marked columns solved in it (1: fields of
                     // up to 2^16 points, 2: always, 0: never)
  int z_p2 = 1;    // float z pass on full columns: pair-granular cp.async tiles (0: the staged kernel)
  int z_tma = 0;  // float z pass: 0 the register-staged kernel; 1 a TMA-using variant (z_tma_ctas)
                  // where the shape allows it; 2 required (shapes it cannot take fail).  The
                  // autotuner times the staged kernel against the variants and keeps the fastest.
  int z_tma_ctas = 4;  // TMA kernel shape: 4 = the persistent register-staged kernel with a tensor
                       // prefetch of each CTA's next tile into L2 (three CTAs per SM, 32-slot tiles);
                       // 1 = tiles copied into shared memory by TMA, one 512-thread CTA per SM,
                       // 32-slot tiles; 2 / 3 = two (128 registers) or three (80) 256-thread CTAs
                       // per SM, 16-slot tiles
  size_t z_smem[2];
  int wblk = 0;  // mixed path: work field in the blocked layout
  // per-pass event records (cans_plan_profile)
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  cudaEvent_t host_ev[2] = {nullptr, nullptr};  // cans_poisson_solve_host: upload done, solve done
  std::vector<int> ev_kind;  // pass kind of record r (events 2r, 2r+1)
  int ev_used = 0;
};

namespace cans {

// The checks of a finished solve, from the norms it accumulated on the device (acc, laid out as the
// plan's acc_d): CANS_ERR_INCOMPATIBLE when the singular column's removed weighted sum exceeds
// compat_tol * compat_scale * ||f||_2; CANS_ERR_NOT_CONVERGED when a norm is not finite, when a
// refinement sweep (from the second on) reduced a residual still above tol by less than half, or
// (verify) when the final relative residual acc[nacc-4] / acc[nacc-3] exceeds tol^2; else CANS_OK.
struct SolveCheck {
  int nacc, sweeps;   // sweeps: refinement sweeps whose residual norms acc[1 .. sweeps] hold
  int compat, verify; // compat: acc[nacc-7] holds the singular column's weighted sum
  double tol, compat_scale, compat_tol;
};

__device__ __forceinline__ int solve_check(const double* acc, const SolveCheck& c) {
  const double ff = acc[0];
  if (c.compat && !(fabs(acc[c.nacc - 7]) <= c.compat_tol * c.compat_scale * sqrt(ff))) return CANS_ERR_INCOMPATIBLE;
  if (!isfinite(ff)) return CANS_ERR_NOT_CONVERGED;
  for (int s = 0; s < c.sweeps; ++s) {
    const double r2 = acc[1 + s];
    if (!isfinite(r2)) return CANS_ERR_NOT_CONVERGED;
    if (s >= 1 && r2 > c.tol * c.tol * ff && r2 > 0.25 * acc[s]) return CANS_ERR_NOT_CONVERGED;
  }
  if (c.verify) {
    const double rr = acc[c.nacc - 4], f2 = acc[c.nacc - 3];
    if (!(rr <= c.tol * c.tol * f2)) return CANS_ERR_NOT_CONVERGED;
  }
  return CANS_OK;
}

// layout of the working field of this plan and precision (the FP64 path works in p: natural)
inline WLay wlay(const cans_plan_s* P, bool working_float) {
  WLay w;
  w.blk = (working_float && P->wblk) ? 1 : 0;
  w.nx = P->n[0];
  w.ny = P->n[1];
  w.nbx = (P->n[0] + 31) / 32;
  return w;
}

// The plan's reproducible block sum (detsum.cuh) into *out (nullptr: no sum).
inline DetSum plan_sum(const cans_plan_s* P, double* out) {
  DetSum d;
  d.slots = P->dsum_slots;
  d.count = P->dsum_count;
  d.out = out;
  return d;
}

// pass launchers (each in its own translation unit)
template <typename T, int MODE>
cudaError_t launch_xfwd(const cans_plan_s* P, const double* f, const float* Phi, const float* Plo, T* dst,
                        double* acc, cudaStream_t st);
// forward x-pass whose input is the divergence of a channel's face velocities (DivArgs), formed on the fly
template <typename T>
cudaError_t launch_xfwd_div(const cans_plan_s* P, const DivArgs& d, T* dst, double* acc, cudaStream_t st);
DivArgs div_args(const cans_plan_s* P, const double* u, const double* v, const double* w, double* fout, double num,
                 const double* dt, double gamma);
template <typename T, int MODE>
cudaError_t launch_xinv(const cans_plan_s* P, const T* src, double* p, float* Phi, float* Plo, double scale,
                        double* gauge, cudaStream_t st);
template <typename T, int DIR>
cudaError_t launch_y(const cans_plan_s* P, T* w, cudaStream_t st);
// part: -1 the whole z pass; in the mixed path 0 = the float columns, 1 = the marked double columns
// compat (optional): receives sum_k dzf_k d_k of the singular column before its projection
template <typename T>
cudaError_t launch_z(const cans_plan_s* P, T* w, const double* gauge, cudaStream_t st, int part = -1,
                     double* compat = nullptr);
// the TMA-fed float z kernel takes this plan's shape and this work field (kern_z.cu)
bool ztma_feasible(const cans_plan_s* P, const void* w);
template <typename T>
cudaError_t launch_zspec(const cans_plan_s* P, T* w, const double* gauge, cudaStream_t st, double* compat = nullptr);
// Fold the checks of a finished solve into the plan's status word (cans_plan_status): one 32-thread
// kernel on the solve's stream; the first error recorded stays until the word is read.  compat: the
// singular column's weighted sum is in acc[nacc-7]; verify: acc[nacc-4], acc[nacc-3] hold ||r||^2,
// ||f||^2 of the result.
cudaError_t launch_solve_status(const cans_plan_s* P, bool compat, bool verify, cudaStream_t st);
SolveCheck solve_check_args(const cans_plan_s* P, bool compat, bool verify);
cudaError_t launch_residual_norms(const cans_plan_s* P, const double* f, const double* p, double* acc2, cudaStream_t st);
cudaError_t launch_weighted_sum(const cans_plan_s* P, const double* f, double* acc2, cudaStream_t st);
cudaError_t launch_momentum(const cans_plan_s* P, const double* u, const double* v, const double* w, const double* p,
                            double* ru, double* rv, double* rw, double* us, double* vs, double* ws, double nu,
                            double alpha, double beta, double gamma, const double* dt_dev, cudaStream_t st,
                            double sigma = 0.0);
cudaError_t launch_divergence(const cans_plan_s* P, const double* u, const double* v, const double* w, double* f,
                              double scale_num, const double* dt_dev, double gamma, int weighted, cudaStream_t st);
cudaError_t launch_correct(const cans_plan_s* P, const double* us, const double* vs, const double* ws,
                           const double* phi, double* u, double* v, double* w, double* p, double gamma,
                           const double* dt_dev, int weighted, double* bulk, cudaStream_t st, double lcoef = 0.0);
cudaError_t launch_forcing(const cans_plan_s* P, double* u, const double* bulk, double ubulk, cudaStream_t st);
cudaError_t launch_chkdt(const cans_plan_s* P, const double* u, const double* v, const double* w,
                         unsigned long long* dti_bits, double* dt_dev, double cfl, double nu, double dt_fixed,
                         cudaStream_t st);

StencilDF stencil_df(const cans_plan_s* P);

// launch shape of a line-transform kernel (lines of N reals, `count` lines or columns, complex
// element size elem2, preferred lines per CTA)
Launch line_launch_shape(int N, int count, size_t elem2, int prefer_nl);
// warp-per-line x-passes of the mixed path (kern_xw.cu); *handled is false when the shape or the
// pointer alignment is not one they take, and the caller then uses the CTA-wide kernels
template <int MODE>
cudaError_t launch_xfwd_warp(const cans_plan_s* P, const double* f, const float* Phi, const float* Plo, float* dst,
                             double* acc, cudaStream_t st, bool* handled);
cudaError_t launch_xfwd_div_warp(const cans_plan_s* P, const DivArgs& d, float* dst, double* acc, cudaStream_t st,
                                 bool* handled);
cudaError_t launch_scale_z(const cans_plan_s* P, const double* in, double* out, const double* wz, cudaStream_t st);
cudaError_t launch_remove_weighted_mean(const cans_plan_s* P, double* f, double* acc2, cudaStream_t st);
cudaError_t launch_residual(const cans_plan_s* P, const double* f, const float* Phi, const float* Plo, bool plo,
                            float* r, double* norm_acc, cudaStream_t st);
bool xres_warp_ok(const cans_plan_s* P, const float* W);
bool xres_cta_ok(const cans_plan_s* P, const float* W);
cudaError_t launch_xfwd32_cta(const cans_plan_s* P, float* W, cudaStream_t st);
cudaError_t launch_xfwd32_warp(const cans_plan_s* P, float* W, cudaStream_t st);
// y-pass with the x-slots across the lanes (kern_yc.cu): taken first where the shape allows it
template <int DIR>
cudaError_t launch_y_cols(const cans_plan_s* P, float* w, cudaStream_t st, bool* handled);
template <int MODE>
cudaError_t launch_xinv_warp(const cans_plan_s* P, const float* src, double* p, float* Phi, float* Plo, double scale,
                             double* gauge, cudaStream_t st, bool* handled);

// NVTX range and, while cans_plan_profile is on, a CUDA event pair on `st` around the launches made
// during its lifetime, recorded as pass kind `kind` (a cans_pass).
struct PassTimer {
  cans_plan_s* P;
  cudaStream_t st;
  int rec = -1;
  PassTimer(cans_plan_s* P, int kind, cudaStream_t st);
  ~PassTimer();
  PassTimer(const PassTimer&) = delete;
  PassTimer& operator=(const PassTimer&) = delete;
};

// Opt a kernel into more than 48 KB of dynamic shared memory.  The attribute is set once per kernel
// and size (remembered per device), so later launches -- including those inside a stream capture --
// make no attribute call.
cudaError_t set_smem(const void* fn, size_t bytes);

template <typename T> const LineTab<T>& tab_x(const cans_plan_s* P);
template <> inline const LineTab<double>& tab_x<double>(const cans_plan_s* P) { return P->tx_d; }
template <> inline const LineTab<float>& tab_x<float>(const cans_plan_s* P) { return P->tx_f; }
template <typename T> const LineTab<T>& tab_y(const cans_plan_s* P);
template <> inline const LineTab<double>& tab_y<double>(const cans_plan_s* P) { return P->ty_d; }
template <> inline const LineTab<float>& tab_y<float>(const cans_plan_s* P) { return P->ty_f; }

// Compile-time FFT lengths (M = N/2) that get specialised kernels; others use the runtime path.
#define CANS_FOR_EACH_M(X) X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(256) X(512)

}  // namespace cans
