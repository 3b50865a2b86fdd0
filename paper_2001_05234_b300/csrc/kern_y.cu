// y-pass of the solver: the transform F^y of Eq. poi_reduced along y, forward or inverse, on tiles
// of nl consecutive x-slots at one z-plane (rows of the tile are contiguous in memory).
#include "plan.cuh"

namespace cans {

constexpr int MAXV = 8;

template <typename T, int DIR, int MC>
__global__ void __launch_bounds__(512, 2) ypass_kernel(T* __restrict__ w, int nx, int ny, int lognl, LineTab<T> tb) {
  typedef typename V2<T>::t C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int nl = 1 << lognl;
  const Lay L{nl};
  const int NY = MC > 0 ? 2 * MC : ny;
  const int i0 = blockIdx.x * nl;
  T* plane = w + (size_t)blockIdx.y * nx * NY;
  T* bufT = reinterpret_cast<T*>(buf);
  for (int e = threadIdx.x; e < nl * NY; e += blockDim.x) {
    const int l = e & (nl - 1), n = e >> lognl;
    const int i = i0 + l;
    const T v = (i < nx) ? plane[(size_t)n * nx + i] : (T)0;
    if (DIR > 0)
      forward_store<T, MC>(buf, L, tb, n, l, v);
    else
      bufT[L.r(n, l)] = v;
  }
  __syncthreads();
  if (DIR > 0)
    line_forward<MAXV, T, MC>(buf, L, lognl, tb);
  else
    line_inverse<MAXV, T, MC>(buf, L, lognl, tb);
  for (int e = threadIdx.x; e < nl * NY; e += blockDim.x) {
    const int l = e & (nl - 1), n = e >> lognl;
    const int i = i0 + l;
    if (i < nx) plane[(size_t)n * nx + i] = (DIR > 0) ? bufT[L.r(n, l)] : inverse_sample<T, MC>(buf, L, tb, n, l);
  }
}

template <typename T, int DIR, int MC>
static cudaError_t y_m(const cans_plan_s* P, T* w, cudaStream_t st) {
  const Launch& L = P->y_l[sizeof(T) == 8 ? 0 : 1];
  cudaError_t e = set_smem((const void*)ypass_kernel<T, DIR, MC>, L.smem);
  if (e != cudaSuccess) return e;
  dim3 grid((P->n[0] + L.nl - 1) / L.nl, P->n[2]);
  ypass_kernel<T, DIR, MC><<<grid, L.threads, L.smem, st>>>(w, P->n[0], P->n[1], L.lognl, tab_y<T>(P));
  return cudaGetLastError();
}

template <typename T, int DIR>
cudaError_t launch_y(const cans_plan_s* P, T* w, cudaStream_t st) {
  if (P->n[1] < 2) return cudaSuccess;
  switch (P->dy.m) {
#define CASE_M(MM) \
  case MM: return y_m<T, DIR, MM>(P, w, st);
    CANS_FOR_EACH_M(CASE_M)
#undef CASE_M
    default: return y_m<T, DIR, 0>(P, w, st);
  }
}

template cudaError_t launch_y<double, 1>(const cans_plan_s*, double*, cudaStream_t);
template cudaError_t launch_y<double, -1>(const cans_plan_s*, double*, cudaStream_t);
template cudaError_t launch_y<float, 1>(const cans_plan_s*, float*, cudaStream_t);
template cudaError_t launch_y<float, -1>(const cans_plan_s*, float*, cudaStream_t);

}  // namespace cans
