// Reporting kernels: ||f - (L_h + shift) p||^2 in FP64 (Eq. poi with a non-uniform z) and the
// dzf-weighted sum of f for the compatibility check of a singular problem (when the caller asks for
// residual norms, or verifies every solve), and the status word's check at the end of every solve.
#include <algorithm>

#include "plan.cuh"
#include "tma.cuh"

namespace cans {

__global__ void residual_norm_kernel(const double* __restrict__ f, const double* __restrict__ p, int nx, int ny, int nz,
                                     int bx, int by, int bz, double idx2, double idy2, const double* __restrict__ sa,
                                     const double* __restrict__ sc, double shift, double* out) {
  const size_t N = (size_t)nx * ny * nz;
  double rr = 0, ff = 0;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((size_t)nx * ny));
    const double pc = p[c];
    auto nb = [&](int bc, bool edge, size_t idx_in, size_t idx_wrap) -> double {
      if (!edge) return p[idx_in];
      if (bc == BC_P) return p[idx_wrap];
      if (bc == BC_NN) return pc;
      return -pc;
    };
    const size_t sy = nx, sz = (size_t)nx * ny;
    const double xm = nb(bc_lo(bx), i == 0, c - 1, c + (nx - 1)), xp = nb(bc_hi(bx), i == nx - 1, c + 1, c - (nx - 1));
    const double ym = nb(bc_lo(by), j == 0, c - sy, c + (ny - 1) * sy);
    const double yp = nb(bc_hi(by), j == ny - 1, c + sy, c - (ny - 1) * sy);
    const double zm = nb(bc_lo(bz), k == 0, c - sz, c + (nz - 1) * sz);
    const double zp = nb(bc_hi(bz), k == nz - 1, c + sz, c - (nz - 1) * sz);
    const double Lp = (xm - 2 * pc + xp) * idx2 + (ym - 2 * pc + yp) * idy2 + sc[k] * (zp - pc) + sa[k] * (zm - pc) +
                      shift * pc;
    const double r = f[c] - Lp;
    rr += r * r;
    ff += f[c] * f[c];
  }
  for (int o = 16; o > 0; o >>= 1) {
    rr += __shfl_xor_sync(0xffffffffu, rr, o);
    ff += __shfl_xor_sync(0xffffffffu, ff, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&out[0], rr);
    atomicAdd(&out[1], ff);
  }
}

__global__ void weighted_sum_kernel(const double* __restrict__ f, int nx, int ny, int nz, const double* __restrict__ dzf,
                                    double* out) {
  const size_t N = (size_t)nx * ny * nz;
  double s = 0, sa = 0;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(c / ((size_t)nx * ny));
    s += dzf[k] * f[c];
    sa += dzf[k] * fabs(f[c]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    sa += __shfl_xor_sync(0xffffffffu, sa, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&out[0], s);
    atomicAdd(&out[1], sa);
  }
}

cudaError_t launch_residual_norms(const cans_plan_s* P, const double* f, const double* p, double* acc2, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(acc2, 0, 2 * sizeof(double), st);
  if (e != cudaSuccess) return e;
  residual_norm_kernel<<<148 * 8, 256, 0, st>>>(f, p, P->n[0], P->n[1], P->n[2], P->bc[0], P->bc[1], P->bc[2], P->idx2,
                                                 P->idy2, P->sa_d, P->sc_d, P->shift, acc2);
  return cudaGetLastError();
}

cudaError_t launch_weighted_sum(const cans_plan_s* P, const double* f, double* acc2, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(acc2, 0, 2 * sizeof(double), st);
  if (e != cudaSuccess) return e;
  weighted_sum_kernel<<<148 * 4, 256, 0, st>>>(f, P->n[0], P->n[1], P->n[2], P->dzf_d, acc2);
  return cudaGetLastError();
}

SolveCheck solve_check_args(const cans_plan_s* P, bool compat, bool verify) {
  SolveCheck c;
  c.nacc = P->nacc;
  c.sweeps = (P->opts.prec == CANS_MIXED) ? P->opts.max_sweeps : 0;
  c.compat = compat ? 1 : 0;
  c.verify = verify ? 1 : 0;
  c.tol = P->opts.tol;
  c.compat_scale = P->compat_scale;
  // the mixed path's singular column comes out of float transforms
  c.compat_tol = (P->opts.prec == CANS_MIXED) ? 1e-5 : 1e-9;
  return c;
}

__global__ void solve_status_kernel(const double* __restrict__ acc, SolveCheck c, int* status) {
  if (threadIdx.x != 0) return;
  const int code = solve_check(acc, c);
  if (code != CANS_OK) atomicCAS(status, CANS_OK, code);
}

cudaError_t launch_solve_status(const cans_plan_s* P, bool compat, bool verify, cudaStream_t st) {
  solve_status_kernel<<<1, 32, 0, st>>>(P->acc_d, solve_check_args(P, compat, verify), P->status_d);
  return cudaGetLastError();
}

// out(i, j, k) = in(i, j, k) * wz[k]: the diagonal z weights around the adjoint solve.
__global__ void scale_z_kernel(const double* __restrict__ in, double* __restrict__ out, size_t plane, size_t n,
                               const double* __restrict__ wz) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x)
    out[c] = in[c] * wz[c / plane];
}

// f -= s / total with s = acc[0] (a dzf-weighted sum computed on the device): removes the weighted mean
__global__ void subtract_mean_kernel(double* __restrict__ f, size_t n, const double* __restrict__ acc,
                                     double inv_total) {
  const double m = acc[0] * inv_total;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x)
    f[c] -= m;
}

cudaError_t launch_remove_weighted_mean(const cans_plan_s* P, double* f, double* acc2, cudaStream_t st) {
  cudaError_t e = launch_weighted_sum(P, f, acc2, st);
  if (e != cudaSuccess) return e;
  const size_t n = (size_t)P->n[0] * P->n[1] * P->n[2];
  double lz = 0;
  for (int k = 0; k < P->n[2]; ++k) lz += P->dzf_h[k];
  const int grid = (int)std::min<size_t>((n + 255) / 256, 148 * 16);
  subtract_mean_kernel<<<grid, 256, 0, st>>>(f, n, acc2, 1.0 / ((double)P->n[0] * P->n[1] * lz));
  return cudaGetLastError();
}

cudaError_t launch_scale_z(const cans_plan_s* P, const double* in, double* out, const double* wz, cudaStream_t st) {
  const size_t plane = (size_t)P->n[0] * P->n[1], n = plane * P->n[2];
  const int grid = (int)std::min<size_t>((n + 255) / 256, 148 * 16);
  scale_z_kernel<<<grid, 256, 0, st>>>(in, out, plane, n, wz);
  return cudaGetLastError();
}

// Element-wise double <-> float conversions of the mixed path (integer-arithmetic versions).
__global__ void split_f64_kernel(const double* __restrict__ x, size_t n, float* rn, float* hi, float* lo,
                                 double* back) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    if (rn) rn[i] = d2f_rn(v);
    const df s = df_split(v);
    if (hi) hi[i] = s.hi;
    if (lo) lo[i] = s.lo;
    if (back) back[i] = df_to_double(s);
  }
}

// One thread waits, with the bounded wait of the TMA-fed z kernels, on a shared-memory transaction
// barrier whose phase completes when its one expected arrival has come and the announced bytes have
// landed.  complete != 0: the thread arrives announcing 0 bytes (the phase completes at once);
// complete == 0: it announces 16 bytes that no copy delivers, so the wait runs out after `polls` polls
// and records CANS_ERR_TIMEOUT in the status word.  No copy is ever in flight.
__global__ void bounded_wait_kernel(int* status, unsigned polls, int complete) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  mbar_arrive_expect_tx(&bar, complete ? 0u : 16u);
  if (!mbar_wait_bounded(&bar, 0, polls)) atomicCAS(status, CANS_OK, CANS_ERR_TIMEOUT);
}

// FP64 fused multiply-add throughput: every thread runs 8 independent chains x <- x * m + c for
// `iters` steps (|m| < 1, so the values stay finite and normal) and stores their sum, which keeps the
// compiler from dropping the work.  2 * 8 * iters FP64 operations per thread.
__global__ void __launch_bounds__(256) fp64_fma_kernel(double* __restrict__ out, unsigned iters) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  double x[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) x[q] = 1.0 + 1e-3 * (double)(q + (t & 7));
  const double m = 0.999999, c = 1e-6;
  for (unsigned i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = fma(x[q], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += x[q];
  out[t] = s;
}

}  // namespace cans

extern "C" int cans_fp64_fma_probe(double* out, size_t n_out, unsigned iters, void* cuda_stream, size_t* flops) {
  int dev = 0, sms = 0;
  if (!out || !flops || iters == 0) return CANS_ERR_ARG;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return CANS_ERR_CUDA;
  const size_t threads = (size_t)sms * 8 * 256;  // eight 256-thread blocks per SM
  if (n_out < threads) return CANS_ERR_ARG;
  cans::fp64_fma_kernel<<<sms * 8, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(out, iters);
  *flops = threads * 16 * (size_t)iters;
  return cudaGetLastError() == cudaSuccess ? CANS_OK : CANS_ERR_CUDA;
}

extern "C" int cans_check_bounded_wait(cans_plan_t plan, unsigned polls, int complete, void* cuda_stream) {
  if (!plan || polls == 0 || polls > (1u << 20)) return CANS_ERR_ARG;
  cans::bounded_wait_kernel<<<1, 32, 0, static_cast<cudaStream_t>(cuda_stream)>>>(plan->status_d, polls, complete);
  return cudaGetLastError() == cudaSuccess ? CANS_OK : CANS_ERR_CUDA;
}

extern "C" int cans_split_f64(const double* x, size_t n, float* rn, float* hi, float* lo, double* back,
                              void* cuda_stream) {
  if (n == 0) return CANS_OK;
  if (!x) return CANS_ERR_ARG;
  const int grid = (int)std::min<size_t>((n + 255) / 256, 148 * 16);
  cans::split_f64_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(x, n, rn, hi, lo, back);
  return cudaGetLastError() == cudaSuccess ? CANS_OK : CANS_ERR_CUDA;
}
