// x-passes of the solver: forward transform along contiguous x lines (fused with the FP64->FP32
// conversion, or with the double-float residual of a refinement sweep) and the inverse transform
// (fused with the normalisation and the update of the iterate).  Transform along x = the operator
// F^x of Eq. poi_reduced.
#include <algorithm>

#include "async.cuh"
#include "plan.cuh"
#include "stencil.cuh"

namespace cans {

constexpr int MAXV = 8;  // complex values per thread per FFT stage

template <typename T> __device__ __forceinline__ T from_double(double x);
template <> __device__ __forceinline__ double from_double<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_double<float>(double x) { return d2f_rn(x); }

__device__ __forceinline__ void block_accumulate(float v, double* dst) {
  __shared__ float red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) atomicAdd(dst, (double)v);
  }
}

// Forward x-pass.  MODE 0: read f (double) -> T.  MODE 1 (T = float): the residual
// f - L_h(Phi + Plo) computed on the fly; MODE 2: the same with Plo known to be zero (first sweep).
// MODE 3: f formed on the fly as the divergence of a channel's face velocities (dv), written to
// dv.fout as well when that is set.
// Output lines go to dst (T) in transform slot order.  norm_acc (optional) receives sum f^2 (MODE 0,
// 3) or sum r^2.
template <typename T, int MODE, int MC>
__global__ void __launch_bounds__(512, 2) xfwd_kernel(const double* __restrict__ f, const float* __restrict__ Phi,
                                                      const float* __restrict__ Plo, T* __restrict__ dst, XArgs a,
                                                      LineTab<T> tb, StencilDF S, double* norm_acc, DivArgs dv) {
  typedef typename V2<T>::t C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int nl = 1 << a.lognl;
  const Lay L{nl};
  const int N = MC > 0 ? 2 * MC : a.nx;
  const int line0 = blockIdx.x * nl;
  const float inv_ny = 1.0f / (float)S.n[1];
  float acc = 0.f;
  const double dscale = (MODE == 3) ? dv.scale() : 0.0;
  // copy-in with U independent loads (or residual evaluations) in flight per thread
  constexpr int U = (MODE == 0) ? 8 : 2;
  const int total = nl * N;
  for (int base = threadIdx.x; base < total; base += U * blockDim.x) {
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = base + u * blockDim.x;
      const int l = e / N, n = e - l * N;
      const int line = line0 + l;
      v[u] = (T)0;
      if (e < total && line < a.nlines) {
        const size_t c = (size_t)line * N + n;
        if (MODE == 0) {
          v[u] = from_double<T>(f[c]);
        } else if (MODE == 3) {
          const int k = (int)(((float)line + 0.5f) * inv_ny);
          const double fv = dv.at(dscale, c, n, line - k * S.n[1], k);
          if (dv.fout != nullptr) dv.fout[c] = fv;
          v[u] = from_double<T>(fv);
        } else {
          // k = line / Ny, exact: (line + 1/2)/Ny stays >= 1/(2 Ny) away from an integer
          const int k = (int)(((float)line + 0.5f) * inv_ny);
          const int j = line - k * S.n[1];
          v[u] = (T)residual_point<MODE == 1>(f, Phi, Plo, S, c, n, j, k);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = base + u * blockDim.x;
      if (e < total) {
        const float vf = (float)v[u];
        acc += vf * vf;
        const int l = e / N;
        forward_store<T, MC>(buf, L, tb, e - l * N, l, v[u]);
      }
    }
  }
  __syncthreads();
  line_forward<MAXV, T, MC>(buf, L, a.lognl, tb);
  const T* bufT = reinterpret_cast<const T*>(buf);
  for (int e = threadIdx.x; e < nl * N; e += blockDim.x) {
    const int l = e / N, s = e - l * N;
    const int line = line0 + l;
    if (line < a.nlines) {
      if (a.w.blk) {
        const int k = (int)(((float)line + 0.5f) * inv_ny);
        dst[a.w.at(s, line - k * a.w.ny, k)] = bufT[L.r(s, l)];
      } else {
        dst[(size_t)line * N + s] = bufT[L.r(s, l)];
      }
    }
  }
  if (norm_acc != nullptr) block_accumulate(acc, norm_acc);
}

// Inverse x-pass.  MODE 0: p (double) = scale * x.  MODE 1: Phi = scale * x (the iterate's tail Plo
// is implicitly zero), and (when gauge.out != nullptr) sum_c dzf_k Phi_c into *gauge.out (a reproducible
// block sum).
// MODE 2: (Phi, Plo) += scale * x (double-float).  MODE 3: p = Phi + Plo + scale * x (double).
// MODE 4, 5: as 2, 3 with the old Plo known to be zero (first sweep).
template <typename T, int MODE, int MC>
__global__ void __launch_bounds__(512, 2) xinv_kernel(const T* __restrict__ src, double* __restrict__ p,
                                                      float* __restrict__ Phi, float* __restrict__ Plo, XArgs a,
                                                      LineTab<T> tb, const float* __restrict__ wz,
                                                      const float* __restrict__ wz_lo, int ny, DetSum gauge) {
  typedef typename V2<T>::t C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int nl = 1 << a.lognl;
  const Lay L{nl};
  const int N = MC > 0 ? 2 * MC : a.nx;
  const int line0 = blockIdx.x * nl;
  T* bufT = reinterpret_cast<T*>(buf);
  const float inv_ny = 1.0f / (float)ny;
  {
    constexpr int U = 8;
    const int total = nl * N;
    for (int base = threadIdx.x; base < total; base += U * blockDim.x) {
      T v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = base + u * blockDim.x;
        const int line = line0 + e / N;
        v[u] = (T)0;
        if (e < total && line < a.nlines) {
          if (a.w.blk) {
            const int k = (int)(((float)line + 0.5f) * inv_ny);
            v[u] = src[a.w.at(e - (e / N) * N, line - k * a.w.ny, k)];
          } else {
            v[u] = src[(size_t)line0 * N + e];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = base + u * blockDim.x;
        if (e < total) {
          const int l = e / N;
          bufT[L.r(e - l * N, l)] = v[u];
        }
      }
    }
  }
  __syncthreads();
  line_inverse<MAXV, T, MC>(buf, L, a.lognl, tb);
  df gacc = df_make(0.f, 0.f);
  for (int e = threadIdx.x; e < nl * N; e += blockDim.x) {
    const int l = e / N, n = e - l * N;
    const int line = line0 + l;
    if (line >= a.nlines) continue;
    const size_t o = (size_t)line * N + n;
    const T v = inverse_sample<T, MC>(buf, L, tb, n, l);
    if (MODE == 0) {
      p[o] = (double)v * a.scale;
    } else if (MODE == 1) {
      const float ph = (float)v * (float)a.scale;
      Phi[o] = ph;
      if (gauge.out != nullptr) {
        const int k = line / ny;
        df t = two_prod(ph, wz[k]);  // ph * dzf_k with dzf_k = wz + wz_lo (double-float weight)
        t.lo = __fmaf_rn(ph, wz_lo[k], t.lo);
        gacc = df_add(gacc, t);
      }
    } else {
      const float d = (float)v * (float)a.scale;
      df s = two_sum(Phi[o], d);
      s = fast_two_sum(s.hi, (MODE <= 3) ? s.lo + Plo[o] : s.lo);
      if (MODE == 2 || MODE == 4) {
        Phi[o] = s.hi;
        Plo[o] = s.lo;
      } else {
        p[o] = df_to_double(s);
      }
    }
  }
  if (MODE == 1 && gauge.out != nullptr) det_sum_finish(block_sum_d((double)gacc.hi + (double)gacc.lo), gauge);
}

// ---- pipelined x-passes -------------------------------------------------------------------------
// A tile is nl consecutive lines, contiguous in memory: it is staged with 16-byte cp.async copies
// into padded shared rows (row stride N + PADE elements spreads the lanes of one sample index over
// the banks) while the previous tile is transformed.  The first FFT stage reads the staged rows
// directly; the post-processing (forward) or last stage (inverse) writes to global memory with
// consecutive threads on consecutive slots of one line.
template <typename S>
__device__ __forceinline__ void stage_lines(S* dst, const S* src, int nl, int N, int pad, int lines_valid) {
  constexpr int V = 16 / sizeof(S);
  const int per_line = N / V;
  for (int e = threadIdx.x; e < nl * per_line; e += blockDim.x) {
    const int l = e / per_line, c = (e - l * per_line) * V;
    S* d = dst + (size_t)l * (N + pad) + c;
    if (l < lines_valid) {
      cp_async16(d, src + (size_t)l * N + c);
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) d[v] = (S)0;
    }
  }
  cp_async_commit();
}

// S = double: f -> float lines (the first pass of a mixed solve).  S = float: a float field transformed
// in place (src == dst: each tile's lines are staged whole before the tile writes them back, and tiles
// share no lines), the residual of a refinement sweep written by the streaming stencil.
template <typename S, int MC>
__global__ void __launch_bounds__(512, 2) xfwd_pipe_kernel(const S* f, float* dst, int nlines, int lognl,
                                                           LineTab<float> tb, double* norm_acc) {
  typedef float2 C;
  constexpr int N = 2 * MC, PAD = 16 / sizeof(S);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nl = 1 << lognl;
  S* raw = reinterpret_cast<S*>(smem_raw);  // [2][nl][N + PAD]
  C* buf = reinterpret_cast<C*>(smem_raw + 2 * (size_t)nl * (N + PAD) * sizeof(S));
  const Lay L{nl};
  const int ntiles = (nlines + nl - 1) / nl;
  float acc = 0.f;
  int t = blockIdx.x;
  if (t < ntiles) stage_lines<S>(raw, f + (size_t)t * nl * N, nl, N, PAD, min(nl, nlines - t * nl));
  for (int it = 0; t < ntiles; t += gridDim.x, ++it) {
    const int slot = it & 1;
    const int tn = t + gridDim.x;
    if (tn < ntiles) {
      stage_lines<S>(raw + (size_t)(slot ^ 1) * nl * (N + PAD), f + (size_t)tn * nl * N, nl, N, PAD,
                     min(nl, nlines - tn * nl));
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const S* src = raw + (size_t)slot * nl * (N + PAD);
    const int line0 = t * nl;
    auto load = [&](int l, int n) -> float {
      float v;
      if constexpr (sizeof(S) == 8)
        v = d2f_rn(src[l * (N + PAD) + n]);
      else
        v = src[l * (N + PAD) + n];
      acc += v * v;
      return v;
    };
    auto store = [&](int l, int s, float v) {
      if (line0 + l < nlines) dst[(size_t)(line0 + l) * N + s] = v;
    };
    line_forward_fused<MAXV, float, MC, true>(buf, L, lognl, tb, load, store);
    __syncthreads();
  }
  if (norm_acc != nullptr) block_accumulate(acc, norm_acc);
}

// Inverse x-pass, pipelined; MODE as xinv_kernel.
template <typename T, int MODE, int MC>
__global__ void __launch_bounds__(512, 2) xinv_pipe_kernel(const T* __restrict__ src, double* __restrict__ p,
                                                           float* __restrict__ Phi, float* __restrict__ Plo,
                                                           int nlines, int lognl, double scale, LineTab<T> tb,
                                                           const float* __restrict__ wz,
                                                           const float* __restrict__ wz_lo, int ny, DetSum gauge) {
  typedef typename V2<T>::t C;
  constexpr int N = 2 * MC, PAD = 16 / sizeof(T);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nl = 1 << lognl;
  T* raw = reinterpret_cast<T*>(smem_raw);  // [2][nl][N + PAD]
  C* buf = reinterpret_cast<C*>(smem_raw + 2 * (size_t)nl * (N + PAD) * sizeof(T));
  const Lay L{nl};
  const int ntiles = (nlines + nl - 1) / nl;
  const float fscale = (float)scale;
  df gacc = df_make(0.f, 0.f);
  int t = blockIdx.x;
  if (t < ntiles) stage_lines<T>(raw, src + (size_t)t * nl * N, nl, N, PAD, min(nl, nlines - t * nl));
  for (int it = 0; t < ntiles; t += gridDim.x, ++it) {
    const int slot = it & 1;
    const int tn = t + gridDim.x;
    if (tn < ntiles) {
      stage_lines<T>(raw + (size_t)(slot ^ 1) * nl * (N + PAD), src + (size_t)tn * nl * N, nl, N, PAD,
                     min(nl, nlines - tn * nl));
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const T* rs = raw + (size_t)slot * nl * (N + PAD);
    const int line0 = t * nl;
    auto loadslot = [&](int l, int s) -> T { return rs[l * (N + PAD) + s]; };
    auto store = [&](int l, int n, T v) {
      const int line = line0 + l;
      if (line >= nlines) return;
      const size_t o = (size_t)line * N + n;
      if (MODE == 0) {
        p[o] = (double)v * scale;
      } else if (MODE == 1) {
        const float ph = (float)v * fscale;
        Phi[o] = ph;
        if (gauge.out != nullptr) {
          const int k = line / ny;
          df tt = two_prod(ph, wz[k]);
          tt.lo = __fmaf_rn(ph, wz_lo[k], tt.lo);
          gacc = df_add(gacc, tt);
        }
      } else {
        const float d = (float)v * fscale;
        df s2 = two_sum(Phi[o], d);
        s2 = fast_two_sum(s2.hi, (MODE <= 3) ? s2.lo + Plo[o] : s2.lo);
        if (MODE == 2 || MODE == 4) {
          Phi[o] = s2.hi;
          Plo[o] = s2.lo;
        } else {
          p[o] = df_to_double(s2);
        }
      }
    };
    line_inverse_fused<MAXV, T, MC, true>(buf, L, lognl, tb, loadslot, store);
    __syncthreads();
  }
  if (MODE == 1 && gauge.out != nullptr) det_sum_finish(block_sum_d((double)gacc.hi + (double)gacc.lo), gauge);
}

template <typename K>
static int persistent_grid(K kernel, int threads, size_t smem, int ntiles) {
  int per_sm = 0, dev = 0, sms = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(1, std::min(ntiles, std::max(per_sm, 1) * sms));
}

StencilDF stencil_df(const cans_plan_s* P) {
  StencilDF S;
  S.idx2.hi = (float)P->idx2;
  S.idx2.lo = (float)(P->idx2 - (double)S.idx2.hi);
  S.xlo = bc_lo(P->bc[0]);
  S.xhi = bc_hi(P->bc[0]);
  S.ylo = bc_lo(P->bc[1]);
  S.yhi = bc_hi(P->bc[1]);
  S.zlo = bc_lo(P->bc[2]);
  S.zhi = bc_hi(P->bc[2]);
  S.shift.hi = (float)P->shift;
  S.shift.lo = (float)(P->shift - (double)S.shift.hi);
  S.idy2.hi = (float)P->idy2;
  S.idy2.lo = (float)(P->idy2 - (double)S.idy2.hi);
  S.sa_hi = P->sa_hi;
  S.sa_lo = P->sa_lo;
  S.sc_hi = P->sc_hi;
  S.sc_lo = P->sc_lo;
  for (int d = 0; d < 3; ++d) {
    S.bc[d] = P->bc[d];
    S.n[d] = P->n[d];
  }
  S.iso = (P->idx2 == P->idy2) ? 1 : 0;
  return S;
}

template <typename T, int MODE, int MC>
static cudaError_t xfwd_m(const cans_plan_s* P, const double* f, const float* Phi, const float* Plo, T* dst,
                          double* acc, cudaStream_t st, const DivArgs* dv = nullptr) {
  const Launch& L = P->x_l[sizeof(T) == 8 ? 0 : 1];
  XArgs a{P->n[0], P->n[1] * P->n[2], L.lognl, 1.0, wlay(P, sizeof(T) == 4)};
  cudaError_t e = set_smem((const void*)xfwd_kernel<T, MODE, MC>, L.smem);
  if (e != cudaSuccess) return e;
  const int grid = (a.nlines + L.nl - 1) / L.nl;
  xfwd_kernel<T, MODE, MC><<<grid, L.threads, L.smem, st>>>(f, Phi, Plo, dst, a, tab_x<T>(P), stencil_df(P), acc,
                                                            dv != nullptr ? *dv : DivArgs{});
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_xfwd_div(const cans_plan_s* P, const DivArgs& d, T* dst, double* acc, cudaStream_t st) {
  if (sizeof(T) == 4) {
    bool handled = false;
    const cudaError_t e = launch_xfwd_div_warp(P, d, reinterpret_cast<float*>(dst), acc, st, &handled);
    if (handled) return e;
  }
  switch (P->dx.m) {
#define CASE_M(MM) \
  case MM: return xfwd_m<T, 3, MM>(P, nullptr, nullptr, nullptr, dst, acc, st, &d);
    CANS_FOR_EACH_M(CASE_M)
#undef CASE_M
    default: return xfwd_m<T, 3, 0>(P, nullptr, nullptr, nullptr, dst, acc, st, &d);
  }
}
template cudaError_t launch_xfwd_div<double>(const cans_plan_s*, const DivArgs&, double*, double*, cudaStream_t);
template cudaError_t launch_xfwd_div<float>(const cans_plan_s*, const DivArgs&, float*, double*, cudaStream_t);

template <typename S, int MC>
static cudaError_t xfwd_pipe_m(const cans_plan_s* P, const S* f, float* dst, double* acc, cudaStream_t st) {
  constexpr int PAD = 16 / sizeof(S);
  Launch L = P->x_l[1];
  size_t smem = L.smem + 2 * (size_t)L.nl * (2 * MC + PAD) * sizeof(S);
  while (smem > (size_t)110 * 1024 && L.nl > 1) {  // keep two CTAs per SM
    L = line_launch_shape(2 * MC, P->n[1] * P->n[2], sizeof(float2), L.nl / 2);
    smem = L.smem + 2 * (size_t)L.nl * (2 * MC + PAD) * sizeof(S);
  }
  cudaError_t e = set_smem((const void*)xfwd_pipe_kernel<S, MC>, smem);
  if (e != cudaSuccess) return e;
  const int nlines = P->n[1] * P->n[2];
  const int grid = persistent_grid(xfwd_pipe_kernel<S, MC>, L.threads, smem, (nlines + L.nl - 1) / L.nl);
  xfwd_pipe_kernel<S, MC><<<grid, L.threads, smem, st>>>(f, dst, nlines, L.lognl, P->tx_f, acc);
  return cudaGetLastError();
}

// The CTA-wide forward x pass of a float field in place (the sweep residual the streaming stencil
// wrote), for x lengths with a compile-time engine, a natural-layout field, 16-byte aligned.
bool xres_cta_ok(const cans_plan_s* P, const float* W) {
  if (P->wblk || (reinterpret_cast<uintptr_t>(W) & 15) != 0) return false;
  switch (P->dx.m) {
#define CASE_M(MM) \
  case MM:         \
    return true;
    CANS_FOR_EACH_M(CASE_M)
#undef CASE_M
    default: return false;
  }
}

cudaError_t launch_xfwd32_cta(const cans_plan_s* P, float* W, cudaStream_t st) {
  switch (P->dx.m) {
#define CASE_M(MM) \
  case MM: return xfwd_pipe_m<float, MM>(P, W, W, nullptr, st);
    CANS_FOR_EACH_M(CASE_M)
#undef CASE_M
    default: return cudaErrorNotSupported;
  }
}

template <typename T, int MODE>
cudaError_t launch_xfwd(const cans_plan_s* P, const double* f, const float* Phi, const float* Plo, T* dst,
                        double* acc, cudaStream_t st) {
  if (sizeof(T) == 4) {
    bool handled = false;
    const cudaError_t e =
        launch_xfwd_warp<MODE>(P, f, Phi, Plo, reinterpret_cast<float*>(dst), acc, st, &handled);
    if (handled) return e;
  }
  // the pipelined kernel stages f with 16-byte copies: f must be 16-byte aligned (lines of N doubles
  // with N even then all are); a double array that is only 8-byte aligned takes the kernel below
  if (MODE == 0 && sizeof(T) == 4 && !P->wblk && (reinterpret_cast<uintptr_t>(f) & 15) == 0) {
    switch (P->dx.m) {
#define CASE_M(MM) \
  case MM: return xfwd_pipe_m<double, MM>(P, f, reinterpret_cast<float*>(dst), acc, st);
      CANS_FOR_EACH_M(CASE_M)
#undef CASE_M
      default: break;
    }
  }
  switch (P->dx.m) {
#define CASE_M(MM) \
  case MM: return xfwd_m<T, MODE, MM>(P, f, Phi, Plo, dst, acc, st);
    CANS_FOR_EACH_M(CASE_M)
#undef CASE_M
    default: return xfwd_m<T, MODE, 0>(P, f, Phi, Plo, dst, acc, st);
  }
}

template <typename T, int MODE, int MC>
static cudaError_t xinv_m(const cans_plan_s* P, const T* src, double* p, float* Phi, float* Plo, double scale,
                          double* gauge, cudaStream_t st) {
  const Launch& L = P->x_l[sizeof(T) == 8 ? 0 : 1];
  XArgs a{P->n[0], P->n[1] * P->n[2], L.lognl, scale, wlay(P, sizeof(T) == 4)};
  cudaError_t e = set_smem((const void*)xinv_kernel<T, MODE, MC>, L.smem);
  if (e != cudaSuccess) return e;
  const int grid = (a.nlines + L.nl - 1) / L.nl;
  if ((size_t)grid > P->dsum_nslots) return cudaErrorInvalidConfiguration;
  xinv_kernel<T, MODE, MC><<<grid, L.threads, L.smem, st>>>(src, p, Phi, Plo, a, tab_x<T>(P), P->dzf_f,
                                                            P->dzf_flo, P->n[1], plan_sum(P, gauge));
  return cudaGetLastError();
}

template <typename T, int MODE, int MC>
static cudaError_t xinv_pipe_m(const cans_plan_s* P, const T* src, double* p, float* Phi, float* Plo, double scale,
                               double* gauge, cudaStream_t st) {
  Launch L = P->x_l[sizeof(T) == 8 ? 0 : 1];
  constexpr int PAD = 16 / sizeof(T);
  size_t smem = L.smem + 2 * (size_t)L.nl * (2 * MC + PAD) * sizeof(T);
  while (smem > (size_t)110 * 1024 && L.nl > 1) {
    L = line_launch_shape(2 * MC, P->n[1] * P->n[2], sizeof(typename V2<T>::t), L.nl / 2);
    smem = L.smem + 2 * (size_t)L.nl * (2 * MC + PAD) * sizeof(T);
  }
  cudaError_t e = set_smem((const void*)xinv_pipe_kernel<T, MODE, MC>, smem);
  if (e != cudaSuccess) return e;
  const int nlines = P->n[1] * P->n[2];
  const int grid = persistent_grid(xinv_pipe_kernel<T, MODE, MC>, L.threads, smem, (nlines + L.nl - 1) / L.nl);
  if ((size_t)grid > P->dsum_nslots) return cudaErrorInvalidConfiguration;
  xinv_pipe_kernel<T, MODE, MC><<<grid, L.threads, smem, st>>>(src, p, Phi, Plo, nlines, L.lognl, scale, tab_x<T>(P),
                                                               P->dzf_f, P->dzf_flo, P->n[1], plan_sum(P, gauge));
  return cudaGetLastError();
}

template <typename T, int MODE>
cudaError_t launch_xinv(const cans_plan_s* P, const T* src, double* p, float* Phi, float* Plo, double scale,
                        double* gauge, cudaStream_t st) {
  if (sizeof(T) == 4) {
    bool handled = false;
    const cudaError_t e = launch_xinv_warp<MODE>(P, reinterpret_cast<const float*>(src), p, Phi, Plo, scale, gauge,
                                                 st, &handled);
    if (handled) return e;
  }
  // the pipelined kernel stages src with 16-byte copies (src is the caller's p in place on the FP64
  // path, which may be only 8-byte aligned)
  if (!(sizeof(T) == 4 && P->wblk) && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
    switch (P->dx.m) {
#define CASE_M(MM) \
  case MM: return xinv_pipe_m<T, MODE, MM>(P, src, p, Phi, Plo, scale, gauge, st);
      CANS_FOR_EACH_M(CASE_M)
#undef CASE_M
      default: break;
    }
  }
  switch (P->dx.m) {
#define CASE_M(MM) \
  case MM: return xinv_m<T, MODE, MM>(P, src, p, Phi, Plo, scale, gauge, st);
    CANS_FOR_EACH_M(CASE_M)
#undef CASE_M
    default: return xinv_m<T, MODE, 0>(P, src, p, Phi, Plo, scale, gauge, st);
  }
}

template cudaError_t launch_xfwd<double, 0>(const cans_plan_s*, const double*, const float*, const float*, double*,
                                            double*, cudaStream_t);
template cudaError_t launch_xfwd<float, 0>(const cans_plan_s*, const double*, const float*, const float*, float*,
                                           double*, cudaStream_t);
template cudaError_t launch_xfwd<float, 1>(const cans_plan_s*, const double*, const float*, const float*, float*,
                                           double*, cudaStream_t);
template cudaError_t launch_xfwd<float, 2>(const cans_plan_s*, const double*, const float*, const float*, float*,
                                           double*, cudaStream_t);
template cudaError_t launch_xinv<double, 0>(const cans_plan_s*, const double*, double*, float*, float*, double, double*,
                                            cudaStream_t);
template cudaError_t launch_xinv<float, 0>(const cans_plan_s*, const float*, double*, float*, float*, double, double*,
                                           cudaStream_t);
template cudaError_t launch_xinv<float, 1>(const cans_plan_s*, const float*, double*, float*, float*, double, double*,
                                           cudaStream_t);
template cudaError_t launch_xinv<float, 2>(const cans_plan_s*, const float*, double*, float*, float*, double, double*,
                                           cudaStream_t);
template cudaError_t launch_xinv<float, 3>(const cans_plan_s*, const float*, double*, float*, float*, double, double*,
                                           cudaStream_t);
template cudaError_t launch_xinv<float, 4>(const cans_plan_s*, const float*, double*, float*, float*, double, double*,
                                           cudaStream_t);
template cudaError_t launch_xinv<float, 5>(const cans_plan_s*, const float*, double*, float*, float*, double, double*,
                                           cudaStream_t);

}  // namespace cans
