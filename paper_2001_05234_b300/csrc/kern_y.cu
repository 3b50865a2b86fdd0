// y-pass of the solver: the transform F^y of Eq. poi_reduced along y, forward or inverse, on tiles
// of nl consecutive x-slots at one z-plane (rows of the tile are contiguous in memory).
#include <algorithm>

#include "async.cuh"
#include "plan.cuh"

namespace cans {

constexpr int MAXV = 8;

template <typename T, int DIR, int MC>
__global__ void __launch_bounds__(512, 2) ypass_kernel(T* __restrict__ w, int nx, int ny, int lognl, LineTab<T> tb,
                                                       WLay wl) {
  typedef typename V2<T>::t C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int nl = 1 << lognl;
  const Lay L{nl};
  const int NY = MC > 0 ? 2 * MC : ny;
  const int i0 = blockIdx.x * nl;
  T* plane = w + wl.ybase(i0, blockIdx.y);  // element (l, j) at plane[j * rs + l]
  const int rs = wl.yrow();
  T* bufT = reinterpret_cast<T*>(buf);
  // copy-in: U independent loads in flight per thread before the shared-memory stores
  constexpr int U = 8;
  const int total = nl * NY;
  for (int base = threadIdx.x; base < total; base += U * blockDim.x) {
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = base + u * blockDim.x;
      const int l = e & (nl - 1), n = e >> lognl;
      v[u] = (e < total && i0 + l < nx) ? plane[(size_t)n * rs + l] : (T)0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = base + u * blockDim.x;
      if (e < total) {
        const int l = e & (nl - 1), n = e >> lognl;
        if (DIR > 0)
          forward_store<T, MC>(buf, L, tb, n, l, v[u]);
        else
          bufT[L.r(n, l)] = v[u];
      }
    }
  }
  __syncthreads();
  if (DIR > 0)
    line_forward<MAXV, T, MC>(buf, L, lognl, tb);
  else
    line_inverse<MAXV, T, MC>(buf, L, lognl, tb);
  for (int e = threadIdx.x; e < nl * NY; e += blockDim.x) {
    const int l = e & (nl - 1), n = e >> lognl;
    const int i = i0 + l;
    if (i < nx) plane[(size_t)n * rs + l] = (DIR > 0) ? bufT[L.r(n, l)] : inverse_sample<T, MC>(buf, L, tb, n, l);
  }
}

// ---- pipelined y-pass ---------------------------------------------------------------------------
// Persistent CTAs walk the tiles (nl consecutive x-slots of one z-plane); the raw rows of tile t + G
// are fetched (cp.async) into the other half of a double buffer while tile t is transformed.
template <typename T, int DIR, int MC>
__global__ void __launch_bounds__(512, 2) ypass_pipe_kernel(T* __restrict__ w, int nx, int nz, int lognl,
                                                            LineTab<T> tb, WLay wl, int vec) {
  typedef typename V2<T>::t C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nl = 1 << lognl;
  const int NY = 2 * MC;
  T* raw = reinterpret_cast<T*>(smem_raw);                             // [2][NY][nl]
  C* buf = reinterpret_cast<C*>(smem_raw + 2 * (size_t)NY * nl * sizeof(T));  // FFT work area
  const Lay L{nl};
  const int tiles_x = (nx + nl - 1) / nl;
  const int ntiles = tiles_x * nz;
  const int rs = wl.yrow();
  auto fetch = [&](int t, int slot) {
    const int i0 = (t % tiles_x) * nl, k = t / tiles_x;
    const T* plane = w + wl.ybase(i0, k);
    T* dst = raw + (size_t)slot * NY * nl;
    constexpr int V = 16 / sizeof(T);
    if (vec && i0 + nl <= nx) {
      const int per_row = nl / V;
      for (int e = threadIdx.x; e < NY * per_row; e += blockDim.x) {
        const int n = e / per_row, q = (e - n * per_row) * V;
        cp_async16(dst + n * nl + q, plane + (size_t)n * rs + q);
      }
    } else {
      for (int e = threadIdx.x; e < NY * nl; e += blockDim.x) {
        const int n = e >> lognl, l = e & (nl - 1);
        if (i0 + l < nx)
          cp_async_elem(dst + e, plane + (size_t)n * rs + l);
        else
          dst[e] = (T)0;
      }
    }
    cp_async_commit();
  };
  int t = blockIdx.x;
  if (t < ntiles) fetch(t, 0);
  for (int it = 0; t < ntiles; t += gridDim.x, ++it) {
    const int slot = it & 1;
    const int tn = t + gridDim.x;
    if (tn < ntiles) {
      fetch(tn, slot ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const T* src = raw + (size_t)slot * NY * nl;
    const int i0 = (t % tiles_x) * nl, k = t / tiles_x;
    T* plane = w + wl.ybase(i0, k);
    auto load = [&](int l, int n) -> T { return src[n * nl + l]; };
    auto store = [&](int l, int n, T v) {
      if (i0 + l < nx) plane[(size_t)n * rs + l] = v;
    };
    if (DIR > 0)
      line_forward_fused<MAXV, T, MC>(buf, L, lognl, tb, load, store);
    else
      line_inverse_fused<MAXV, T, MC>(buf, L, lognl, tb, load, store);
    __syncthreads();  // the work area and this raw slot are reused by the next tile
  }
}

template <typename T, int DIR, int MC>
static cudaError_t ypipe_m(const cans_plan_s* P, T* w, cudaStream_t st) {
  const Launch& L = P->y_l[sizeof(T) == 8 ? 0 : 1];
  const size_t smem = L.smem + 2 * (size_t)P->n[1] * L.nl * sizeof(T);
  cudaError_t e = set_smem((const void*)ypass_pipe_kernel<T, DIR, MC>, smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ypass_pipe_kernel<T, DIR, MC>, L.threads, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int ntiles = ((P->n[0] + L.nl - 1) / L.nl) * P->n[2];
  const int grid = std::max(1, std::min(ntiles, std::max(per_sm, 1) * sms));
  const WLay wl = wlay(P, sizeof(T) == 4);
  const int vec = ((wl.blk || P->n[0] % 4 == 0) && (reinterpret_cast<uintptr_t>(w) & 15) == 0) ? 1 : 0;
  ypass_pipe_kernel<T, DIR, MC><<<grid, L.threads, smem, st>>>(w, P->n[0], P->n[2], L.lognl, tab_y<T>(P), wl, vec);
  return cudaGetLastError();
}

template <typename T, int DIR, int MC>
static cudaError_t y_m(const cans_plan_s* P, T* w, cudaStream_t st) {
  const Launch& L = P->y_l[sizeof(T) == 8 ? 0 : 1];
  cudaError_t e = set_smem((const void*)ypass_kernel<T, DIR, MC>, L.smem);
  if (e != cudaSuccess) return e;
  dim3 grid((P->n[0] + L.nl - 1) / L.nl, P->n[2]);
  ypass_kernel<T, DIR, MC><<<grid, L.threads, L.smem, st>>>(w, P->n[0], P->n[1], L.lognl, tab_y<T>(P),
                                                            wlay(P, sizeof(T) == 4));
  return cudaGetLastError();
}

template <typename T, int DIR>
cudaError_t launch_y(const cans_plan_s* P, T* w, cudaStream_t st) {
  if (P->n[1] < 2) return cudaSuccess;
  if (sizeof(T) == 4) {
    bool handled = false;
    const cudaError_t e = launch_y_cols<DIR>(P, reinterpret_cast<float*>(w), st, &handled);
    if (handled) return e;
  }
  switch (P->dy.m) {
#define CASE_M(MM) \
  case MM: return ypipe_m<T, DIR, MM>(P, w, st);
    CANS_FOR_EACH_M(CASE_M)
#undef CASE_M
    default: return y_m<T, DIR, 0>(P, w, st);
  }
}

// Periodic (uniform) z: the z operator is diagonalised too.  A CTA takes nl consecutive x-slots of one
// y-slot, transforms each column along z (real DFT), divides slot s by mu_x(i) + mu_y(j) + mu_z(s)
// (+ the Helmholtz shift),
// and transforms back (scaled by 1/Nz).  The singular (0,0,0) mode gets Nz * target, which makes the
// column mean `target` (0, or the gauge correction of the mixed path's first sweep).
template <typename T, int MC>
__global__ void __launch_bounds__(512, 2) zspec_kernel(T* __restrict__ w, int nx, int ny, int nz, int lognl,
                                                       LineTab<T> tb, const T* __restrict__ mux,
                                                       const T* __restrict__ muy, const T* __restrict__ muz,
                                                       int singular, const double* gauge, double gauge_scale,
                                                       T shift, WLay wl, double* compat, double cw) {
  typedef typename V2<T>::t C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int nl = 1 << lognl;
  const Lay L{nl};
  const int NZ = MC > 0 ? 2 * MC : nz;
  const int i0 = blockIdx.x * nl, j = blockIdx.y;
  const size_t plane = wl.zstride();
  T* col0 = w + wl.zbase(i0, j);
  T* bufT = reinterpret_cast<T*>(buf);
  constexpr int U = 8;
  const int total = nl * NZ;
  for (int base = threadIdx.x; base < total; base += U * blockDim.x) {
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = base + u * blockDim.x;
      const int l = e & (nl - 1), n = e >> lognl;
      v[u] = (e < total && i0 + l < nx) ? col0[(size_t)n * plane + l] : (T)0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = base + u * blockDim.x;
      if (e < total) forward_store<T, MC>(buf, L, tb, e >> lognl, e & (nl - 1), v[u]);
    }
  }
  __syncthreads();
  line_forward<MAXV, T, MC>(buf, L, lognl, tb);
  const T my = muy[j] + shift;
  for (int e = threadIdx.x; e < nl * NZ; e += blockDim.x) {
    const int l = e & (nl - 1), s = e >> lognl;
    const int i = i0 + l;
    if (i >= nx) continue;
    T v = bufT[L.r(s, l)];
    if (singular && i == 0 && j == 0 && s == 0) {
      if (compat != nullptr) *compat = cw * (double)v;  // uniform z: sum_k dz d_k = dz * slot 0
      v = (gauge != nullptr) ? (T)(gauge_scale * (*gauge) * NZ) : (T)0;
    }
    else
      v = v / (mux[i] + my + muz[s]);
    bufT[L.r(s, l)] = v;
  }
  __syncthreads();
  line_inverse<MAXV, T, MC>(buf, L, lognl, tb);
  const T inv = (T)1 / (T)NZ;
  for (int e = threadIdx.x; e < nl * NZ; e += blockDim.x) {
    const int l = e & (nl - 1), n = e >> lognl;
    if (i0 + l < nx) col0[(size_t)n * plane + l] = inverse_sample<T, MC>(buf, L, tb, n, l) * inv;
  }
}

template <typename T> const LineTab<T>& tab_z(const cans_plan_s* P);
template <> const LineTab<double>& tab_z<double>(const cans_plan_s* P) { return P->tz_d; }
template <> const LineTab<float>& tab_z<float>(const cans_plan_s* P) { return P->tz_f; }

template <typename T, int MC>
static cudaError_t zspec_m(const cans_plan_s* P, T* w, const double* gauge, cudaStream_t st, double* compat) {
  const Launch& L = P->zs_l[sizeof(T) == 8 ? 0 : 1];
  cudaError_t e = set_smem((const void*)zspec_kernel<T, MC>, L.smem);
  if (e != cudaSuccess) return e;
  dim3 grid((P->n[0] + L.nl - 1) / L.nl, P->n[1]);
  const T* mux = sizeof(T) == 8 ? (const T*)P->mux_d : (const T*)P->mux_f;
  const T* muy = sizeof(T) == 8 ? (const T*)P->muy_d : (const T*)P->muy_f;
  const T* muz = sizeof(T) == 8 ? (const T*)P->muz_d : (const T*)P->muz_f;
  zspec_kernel<T, MC><<<grid, L.threads, L.smem, st>>>(w, P->n[0], P->n[1], P->n[2], L.lognl, tab_z<T>(P), mux, muy,
                                                       muz, P->singular ? 1 : 0, gauge, P->gauge_scale,
                                                       (T)P->shift, wlay(P, sizeof(T) == 4), compat,
                                                       P->dzf_h.empty() ? 0.0 : P->dzf_h[0]);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_zspec(const cans_plan_s* P, T* w, const double* gauge, cudaStream_t st, double* compat) {
  switch (P->dz.m) {
#define CASE_M(MM) \
  case MM: return zspec_m<T, MM>(P, w, gauge, st, compat);
    CANS_FOR_EACH_M(CASE_M)
#undef CASE_M
    default: return zspec_m<T, 0>(P, w, gauge, st, compat);
  }
}

template cudaError_t launch_zspec<double>(const cans_plan_s*, double*, const double*, cudaStream_t, double*);
template cudaError_t launch_zspec<float>(const cans_plan_s*, float*, const double*, cudaStream_t, double*);

template cudaError_t launch_y<double, 1>(const cans_plan_s*, double*, cudaStream_t);
template cudaError_t launch_y<double, -1>(const cans_plan_s*, double*, cudaStream_t);
template cudaError_t launch_y<float, 1>(const cans_plan_s*, float*, cudaStream_t);
template cudaError_t launch_y<float, -1>(const cans_plan_s*, float*, cudaStream_t);

}  // namespace cans
