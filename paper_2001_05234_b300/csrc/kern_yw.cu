// y-pass of the mixed path on the warp-per-line engine (float work field, Ny = 2M with M in
// {128, 256, 512}, Nx a multiple of 16): the transform F^y of Eq. poi_reduced, forward or inverse.
//
// A persistent CTA of 16 warps walks tiles of 16 consecutive x-slots x Ny rows of one z-plane.  A
// tile is fetched with 4-byte cp.async copies into a row-pair layout T[m][l] = (x[2m][l], x[2m+1][l])
// of float2 with a row stride of 17 cells, so that a warp walking one column with its lanes along m
// touches 16 different bank pairs.  Warp w transforms column w in place, using the column itself as
// its exchange buffer; the CTA then writes the tile back in 64-byte row segments.  Two tile buffers:
// the next tile's copies are in flight while the current one is transformed.
#include <algorithm>

#include "async.cuh"
#include "plan.cuh"
#include "wline.cuh"

namespace cans {
namespace {

constexpr int YW_L = 16;   // x-slots (lines) per tile = warps per CTA
constexpr int YW_RS = 17;  // float2 cells per tile row

struct ColSrc {  // column w of the tile: sample n = T[n/2][w].(n&1)
  const float* c;  // &T[0][w] as floats
  __device__ __forceinline__ float2 pair(int n) { return *reinterpret_cast<const float2*>(c + n * YW_RS); }
  __device__ __forceinline__ float one(int n) { return c[(n >> 1) * (2 * YW_RS) + (n & 1)]; }
  __device__ __forceinline__ float get(int s) { return one(s); }
  __device__ __forceinline__ float2 get2(int s) { return pair(s); }  // slots s, s+1 (s even)
};
struct ColSnk {
  float* c;
  __device__ __forceinline__ void put(int s, float y) { c[(s >> 1) * (2 * YW_RS) + (s & 1)] = y; }
  __device__ __forceinline__ void put2(int s, float a, float b) { pair(s, a, b); }  // s even
  __device__ __forceinline__ void one(int n, float y) { put(n, y); }
  __device__ __forceinline__ void pair(int n, float a, float b) {
    *reinterpret_cast<float2*>(c + n * YW_RS) = make_float2(a, b);
  }
};

// One CTA of 16 warps per SM, one column per warp, two tile buffers: the copies of tile t + G run
// while tile t is transformed.
template <int M, int BC, int DIR>
__global__ void __launch_bounds__(32 * YW_L, 1) yw_kernel(float* __restrict__ w, int nx, int nz, LineTab<float> tb) {
  constexpr int NY = 2 * M, NT = 32 * YW_L;
  constexpr int TILE = M * YW_RS * 2;  // floats per tile buffer
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* T = reinterpret_cast<float*>(smem_raw);  // [2][M][YW_RS] float2
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int tiles_x = nx / YW_L, ntiles = tiles_x * nz;
  const size_t plane = (size_t)nx * NY;
  // copy roles: thread -> column cl and rows n = r0 + RPP q; tile offset so + q * SSTEP, global offset
  // go + q * RPP nx
  constexpr int RPP = NT / YW_L;  // rows per copy pass
  static_assert(NY % RPP == 0 && RPP % 2 == 0, "rows per copy pass");
  const int cl = threadIdx.x & (YW_L - 1), r0 = threadIdx.x / YW_L;
  const int so = (r0 >> 1) * (2 * YW_RS) + 2 * cl + (r0 & 1);
  const size_t go = (size_t)r0 * nx + cl, gstep = (size_t)RPP * nx;
  constexpr int SSTEP = (RPP / 2) * 2 * YW_RS;
  auto tile_base = [&](int t) { return w + (size_t)(t / tiles_x) * plane + (t % tiles_x) * YW_L; };
  auto fetch = [&](int t, float* buf) {
    const float* gp = tile_base(t) + go;
#pragma unroll 8
    for (int q = 0; q < NY / RPP; ++q, gp += gstep) cp_async4(buf + so + q * SSTEP, gp);
    cp_async_commit();
  };
  int t = blockIdx.x;
  if (t < ntiles) fetch(t, T);
  for (int it = 0; t < ntiles; t += gridDim.x, ++it) {
    float* cur = T + (it & 1) * TILE;
    __syncthreads();  // the other buffer's previous tile has been written back
    const int tn = t + gridDim.x;
    if (tn < ntiles) {
      fetch(tn, T + ((it + 1) & 1) * TILE);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    {
      float* col = cur + 2 * wid;
      ColSrc src{col};
      ColSnk snk{col};
      const wl::Strided<YW_RS> xb{reinterpret_cast<float2*>(col)};
      if (DIR > 0)
        wl::forward<M, BC, true, 1, true>(xb, tb, lane, src, snk);
      else
        wl::inverse<M, BC, false, 1, true>(xb, tb, lane, src, snk);
    }
    __syncthreads();
    float* gp = tile_base(t) + go;
#pragma unroll 8
    for (int q = 0; q < NY / RPP; ++q, gp += gstep) *gp = cur[so + q * SSTEP];
  }
}

template <int M, int BC, int DIR>
cudaError_t yw(const cans_plan_s* P, float* w, cudaStream_t st) {
  auto k = yw_kernel<M, BC, DIR>;
  const size_t smem = (size_t)2 * M * YW_RS * sizeof(float2);
  cudaError_t e = set_smem((const void*)k, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * YW_L, smem);
  const int ntiles = (P->n[0] / YW_L) * P->n[2];
  k<<<std::max(1, std::min(ntiles, std::max(per_sm, 1) * sms)), 32 * YW_L, smem, st>>>(w, P->n[0], P->n[2], P->ty_f);
  return cudaGetLastError();
}

}  // namespace

template <int DIR>
cudaError_t launch_y_warp(const cans_plan_s* P, float* w, cudaStream_t st, bool* handled) {
  *handled = false;
  if (P->wblk || P->n[0] % YW_L != 0 || (reinterpret_cast<uintptr_t>(w) & 15)) return cudaSuccess;
  const int bc = P->bc[1];
  *handled = true;
#define YW_CASE(MM)                                                  \
  if (P->dy.m == MM) {                                               \
    if (bc == BC_P) return yw<MM, BC_P, DIR>(P, w, st);              \
    if (bc == BC_NN) return yw<MM, BC_NN, DIR>(P, w, st);            \
    if (bc == BC_ND) return yw<MM, BC_ND, DIR>(P, w, st);            \
    if (bc == BC_DN) return yw<MM, BC_DN, DIR>(P, w, st);            \
    return yw<MM, BC_DD, DIR>(P, w, st);                             \
  }
  YW_CASE(128)
  YW_CASE(256)
  YW_CASE(512)
#undef YW_CASE
  *handled = false;
  return cudaSuccess;
}

template cudaError_t launch_y_warp<1>(const cans_plan_s*, float*, cudaStream_t, bool*);
template cudaError_t launch_y_warp<-1>(const cans_plan_s*, float*, cudaStream_t, bool*);

}  // namespace cans
