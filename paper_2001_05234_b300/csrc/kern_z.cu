// z-pass of the solver: one tridiagonal solve along z per (x, y) mode (Eq. poi_reduced).
//   zpass_f32_kernel : float columns of the mixed path (skips the columns the plan marks as double).
//   zpass_f64_kernel : double columns -- every column of the FP64 path, or the marked low-|mu|
//                      columns of the mixed path (including the singular (0,0) mode), over the
//                      bounding box of the marked columns only.
#include <cstdlib>
#include <mutex>

#include "async.cuh"
#include "plan.cuh"
#include "tma.cuh"

namespace cans {

// Coalesced copy of a TI x Nz tile (TI consecutive x-slots of one y-slot, all z) into the swizzled
// shared layout and back.  Rows are TI elements long; 16-byte vectors when the grid allows it.
template <typename T, typename ZS>
__device__ __forceinline__ void tile_load(T* tile, const T* col0, size_t plane, const ZS& Z, int nz, int ncols,
                                          bool vec) {
  const int TI = Z.ti();
  constexpr int V = 16 / sizeof(T);
  if (vec && ncols == TI) {
    // 16-byte vectors, four in flight per thread before the shared-memory stores
    const int per_row = TI / V;
    const int total = per_row * nz;
    constexpr int U = 4;
    for (int base = threadIdx.x; base < total; base += U * blockDim.x) {
      float4 raw[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = base + u * blockDim.x;
        if (e < total) {
          const int k = e / per_row, q = (e - k * per_row) * V;
          raw[u] = *reinterpret_cast<const float4*>(col0 + (size_t)k * plane + q);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = base + u * blockDim.x;
        if (e < total) {
          const int k = e / per_row, q = (e - k * per_row) * V;
          if (V == 4) {
            const float vv[4] = {raw[u].x, raw[u].y, raw[u].z, raw[u].w};
#pragma unroll
            for (int w = 0; w < 4; ++w) tile[Z.at(k, q + w)] = (T)vv[w];
          } else {
            const double2 v = *reinterpret_cast<const double2*>(&raw[u]);
            tile[Z.at(k, q)] = (T)v.x;
            tile[Z.at(k, q + 1)] = (T)v.y;
          }
        }
      }
    }
  } else {
    for (int e = threadIdx.x; e < TI * nz; e += blockDim.x) {
      const int k = e / TI, ii = e - k * TI;
      if (ii < ncols) tile[Z.at(k, ii)] = col0[(size_t)k * plane + ii];
    }
  }
}

template <typename T, typename ZS>
__device__ __forceinline__ void tile_store(const T* tile, T* col0, size_t plane, const ZS& Z, int nz, int ncols,
                                           bool vec) {
  const int TI = Z.ti();
  constexpr int V = 16 / sizeof(T);
  if (vec && ncols == TI) {
    const int per_row = TI / V;
    for (int e = threadIdx.x; e < per_row * nz; e += blockDim.x) {
      const int k = e / per_row, q = (e - k * per_row) * V;
      T* dst = col0 + (size_t)k * plane + q;
      if (V == 4) {
        float4 v;
        v.x = (float)tile[Z.at(k, q)];
        v.y = (float)tile[Z.at(k, q + 1)];
        v.z = (float)tile[Z.at(k, q + 2)];
        v.w = (float)tile[Z.at(k, q + 3)];
        *reinterpret_cast<float4*>(dst) = v;
      } else {
        double2 v;
        v.x = (double)tile[Z.at(k, q)];
        v.y = (double)tile[Z.at(k, q + 1)];
        *reinterpret_cast<double2*>(dst) = v;
      }
    }
  } else {
    for (int e = threadIdx.x; e < TI * nz; e += blockDim.x) {
      const int k = e / TI, ii = e - k * TI;
      if (ii < ncols) col0[(size_t)k * plane + ii] = tile[Z.at(k, ii)];
    }
  }
}

// The float columns of one staged tile (x-slots i0 .. i0+ncols-1 of y-slot j), one warp per column
// or column pair.  PAIR: x periodic, so x-slots 2q and 2q+1 (q >= 1) share their eigenvalue; a warp
// solves such a pair with one factorisation (zsolve_pair) unless the plan marks one of the two as a
// double column.  Columns the plan marks are left for the double kernel.
template <int MMAX, bool PAIR, typename ZS>
__device__ __forceinline__ void solve_tile_f32(float* tile, const ZS& Z, const ZArgs& a, int i0, int j, int ncols,
                                               const float* sa, const float* sb, const float* sc) {
  constexpr bool CL = MMAX >= 4;  // lane-contiguous coefficient rows, four per 16-byte load
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const float muy = a.muy_f[j] + (float)a.shift;
  auto single = [&](int cidx) {
    const int i = i0 + cidx;
    if (a.mask != nullptr && a.mask[(size_t)j * a.nx + i]) return;
    if (a.nz == 32 * MMAX)
      zsolve_column<MMAX, float, float, false, ZS, true, CL>(tile, cidx, Z, a.nz, a.mux_f[i] + muy, sa, sb, sc,
                                                             nullptr, 0.f);
    else
      zsolve_column<MMAX, float, float, false, ZS, false, CL>(tile, cidx, Z, a.nz, a.mux_f[i] + muy, sa, sb, sc,
                                                              nullptr, 0.f);
  };
  if constexpr (PAIR) {  // i0 and ncols are even (checked at launch)
    for (int q = warp; 2 * q < ncols; q += nwarps) {
      const int c0 = 2 * q, i = i0 + c0;
      const bool m0 = a.mask != nullptr && a.mask[(size_t)j * a.nx + i];
      const bool m1 = a.mask != nullptr && a.mask[(size_t)j * a.nx + i + 1];
      if (i == 0 || m0 || m1) {  // slots 0 and 1 (X_0, X_M) differ; a marked column goes to the double kernel
        single(c0);
        single(c0 + 1);
      } else if (a.nz == 32 * MMAX) {
        zsolve_pair<MMAX, float, float, ZS, true, CL>(tile, c0, c0 + 1, Z, a.nz, a.mux_f[i] + muy, sa, sb, sc);
      } else {
        zsolve_pair<MMAX, float, float, ZS, false, CL>(tile, c0, c0 + 1, Z, a.nz, a.mux_f[i] + muy, sa, sb, sc);
      }
    }
  } else {
    for (int cidx = warp; cidx < ncols; cidx += nwarps) single(cidx);
  }
}

// The marked (low-|mu|, singular) columns of a staged float tile solved in FP64 in place: the body of
// zpass_f64_kernel on a tile already in shared memory (double coefficient rows in sa .. sc).
template <int MMAX, typename ZS>
__device__ __forceinline__ void solve_tile_marked_f64(float* tile, const ZS& Z, const ZArgs& a, int i0, int j,
                                                      int ncols, const double* sa, const double* sb,
                                                      const double* sc) {
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const double muy = a.muy_d[j] + a.shift;
  auto marked = [&](int i) { return a.mask[(size_t)j * a.nx + i] != 0; };
  auto single = [&](int cidx) {
    const int i = i0 + cidx;
    if (!marked(i)) return;
    const double mu = a.mux_d[i] + muy;
    if (a.singular && i == 0 && j == 0) {
      const double target = (a.gauge != nullptr) ? a.gauge_scale * (*a.gauge) : 0.0;
      zsolve_column<MMAX, double, float, true>(tile, cidx, Z, a.nz, mu, sa, sb, sc, a.dzf, target, a.compat);
    } else {
      zsolve_column<MMAX, double, float, false>(tile, cidx, Z, a.nz, mu, sa, sb, sc, nullptr, 0.0);
    }
  };
  if (MMAX >= 2 && a.xpairs) {
    for (int q = warp; 2 * q < ncols; q += nwarps) {
      const int c0 = 2 * q, i = i0 + c0;
      if (i == 0 || !marked(i) || !marked(i + 1)) {
        single(c0);
        single(c0 + 1);
      } else if constexpr (MMAX >= 2) {
        zsolve_pair<MMAX, double, float, ZS, false, false>(tile, c0, c0 + 1, Z, a.nz, a.mux_d[i] + muy, sa, sb, sc);
      }
    }
  } else {
    for (int cidx = warp; cidx < ncols; cidx += nwarps) single(cidx);
  }
}

// F64: the tile's marked columns are solved here in FP64 as well (short columns, MMAX <= 4), so the
// separate double kernel is not launched; sd holds their double coefficient rows.
template <int MMAX, int TIC, bool PAIR, bool F64 = false>
__global__ void __launch_bounds__(256, 3) zpass_f32_kernel(float* __restrict__ w, ZArgs a, ZTab<float> zf,
                                                                      int vec, WLay wl, ZTab<double> zd = {}) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int TI = TIC > 0 ? TIC : a.ti, m = a.m;
  constexpr bool CL = MMAX >= 4;
  const int rs = CL ? 32 * (m + 4) : 32 * m;
  float* sa = reinterpret_cast<float*>(smem_raw);
  float* sb = sa + rs;
  float* sc = sb + rs;
  float* tile = sc + rs;
  const int i0 = blockIdx.x * TI, j = blockIdx.y;
  const size_t plane = wl.zstride();
  float* col0 = w + wl.zbase(i0, j);
  const int ncols = min(TI, a.nx - i0);
  const auto Z = make_zswz<TIC, MMAX>(TI, m);
  stage_zrows<CL>(sa, sb, sc, zf, a.nz, m);
  // the double rows after the tile (8-byte aligned: the tile holds TI * Nz floats, TI even)
  double* da = reinterpret_cast<double*>(tile + (size_t)TI * a.nz + ((TI * a.nz) & 1));
  bool any64 = false;
  if constexpr (F64) {  // does the tile hold a marked column? (a vote, uniform over the CTA)
    any64 = __syncthreads_or((int)threadIdx.x < ncols && a.mask[(size_t)j * a.nx + i0 + threadIdx.x] != 0) != 0;
    if (any64) stage_zrows<false>(da, da + 32 * m, da + 64 * m, zd, a.nz, m);
  }
  tile_load<float>(tile, col0, plane, Z, a.nz, ncols, vec != 0);
  __syncthreads();
  solve_tile_f32<MMAX, PAIR>(tile, Z, a, i0, j, ncols, sa, sb, sc);
  if constexpr (F64) {
    if (any64) solve_tile_marked_f64<MMAX>(tile, Z, a, i0, j, ncols, da, da + 32 * m, da + 64 * m);
  }
  __syncthreads();
  tile_store<float>(tile, col0, plane, Z, a.nz, ncols, vec != 0);
}

// Per-warp values of the two column pairs a warp solves in a pair-granular tile (x-slots i0 .. i0 + 31 of
// y-slot j; 8 warps, pairs q = warp and warp + 8): read from global memory before the tile barrier.
struct PairMu {
  float mu[2][2];
  bool skip[2][2];  // the column is the double kernel's
  bool single[2];   // solve the two columns one by one (slots 0, 1 of x, or a marked column)
};
__device__ __forceinline__ PairMu pair_mu(const ZArgs& a, int i0, int j) {
  PairMu v;
  const int warp = threadIdx.x >> 5;
  const float muy = a.muy_f[j] + (float)a.shift;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int i = i0 + 2 * (warp + 8 * h);
    const bool m0 = a.mask != nullptr && a.mask[(size_t)j * a.nx + i];
    const bool m1 = a.mask != nullptr && a.mask[(size_t)j * a.nx + i + 1];
    v.mu[h][0] = a.mux_f[i] + muy;
    v.mu[h][1] = a.mux_f[i + 1] + muy;
    v.skip[h][0] = m0;
    v.skip[h][1] = m1;
    v.single[h] = i == 0 || m0 || m1;
  }
  return v;
}

// The column pairs of one pair-granular tile, one warp per pair (256 threads): slots 0 and 1 of x
// (X_0, X_M: different eigenvalues) as single columns, a column the plan marks for the double kernel
// skipped, every other pair by zsolve_pair2.
// PAIR false (x not periodic): every column is solved on its own (zsolve_column; its 4-byte accesses
// of the pair-granular tile meet 2-way bank conflicts, lanes l and l + 16).
template <int MMAX, bool PAIR>
__device__ __forceinline__ void solve_tile_p2(float* tile, const ZArgs& a, const PairMu& v, const float* sa,
                                              const float* sb, const float* sc) {
  const ZSwzP<MMAX> Z;
  const int warp = threadIdx.x >> 5;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int c0 = 2 * (warp + 8 * h);
    if (!PAIR || v.single[h]) {
      if (!v.skip[h][0])
        zsolve_column<MMAX, float, float, false, ZSwzP<MMAX>, true, true>(tile, c0, Z, a.nz, v.mu[h][0], sa, sb, sc,
                                                                          nullptr, 0.f);
      if (!v.skip[h][1])
        zsolve_column<MMAX, float, float, false, ZSwzP<MMAX>, true, true>(tile, c0 + 1, Z, a.nz, v.mu[h][1], sa, sb,
                                                                          sc, nullptr, 0.f);
    } else {
      zsolve_pair2<MMAX>(tile, c0, Z, v.mu[h][0], sa, sb, sc);
    }
  }
}

// The float z pass on pair-granular tiles (ZSwzP) for a periodic x direction: full columns
// (Nz = 32 MMAX, MMAX >= 4), tiles of 32 x-slots of a natural-layout field.  The tile arrives by
// 8-byte cp.async copies straight into its swizzled place -- a CTA has all 64 KB of its tile in
// flight at once and holds no registers for it -- and each column pair is solved by zsolve_pair2,
// with both right-hand sides of a row in one 8-byte word.  Same arithmetic per column as
// zpass_f32_kernel (bit-identical results); slot 0 and 1 of x and the columns the plan marks for the
// double kernel are handled as there.
template <int MMAX, bool PAIR>
__global__ void __launch_bounds__(256, 3) zpass_p2_kernel(float* __restrict__ w, ZArgs a, ZTab<float> zf, WLay wl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int TI = 32, rs = 32 * (MMAX + 4);
  float* sa = reinterpret_cast<float*>(smem_raw);
  float* sb = sa + rs;
  float* sc = sb + rs;
  float* tile = sc + rs;
  const int i0 = blockIdx.x * TI, j = blockIdx.y;
  const size_t plane = wl.zstride();
  float* col0 = w + wl.zbase(i0, j);
  const ZSwzP<MMAX> Z;
  {  // thread t copies pair t & 15 of rows (t >> 4) + 16 u
    const int p2 = 2 * (threadIdx.x & 15);
    for (int k = threadIdx.x >> 4; k < 32 * MMAX; k += blockDim.x >> 4) {
      cp_async8(tile + Z.at(k, p2), col0 + (size_t)k * plane + p2);
    }
    cp_async_commit();
  }
  stage_zrows<true>(sa, sb, sc, zf, a.nz, MMAX);
  const PairMu v = pair_mu(a, i0, j);  // global reads in flight with the tile copy
  cp_async_wait<0>();
  __syncthreads();
  solve_tile_p2<MMAX, PAIR>(tile, a, v, sa, sb, sc);
  __syncthreads();
  {  // thread t writes floats 4 (t & 7) .. 4 (t & 7) + 3 of rows (t >> 3) + 32 u
    const int q = 4 * (threadIdx.x & 7);
    for (int k = threadIdx.x >> 3; k < 32 * MMAX; k += blockDim.x >> 3) {
      const float2 lo = *reinterpret_cast<const float2*>(tile + Z.at(k, q));
      const float2 hi = *reinterpret_cast<const float2*>(tile + Z.at(k, q + 2));
      *reinterpret_cast<float4*>(col0 + (size_t)k * plane + q) = make_float4(lo.x, lo.y, hi.x, hi.y);
    }
  }
}

// The float z pass fed by TMA, for full columns (Nz = 32 MMAX, MMAX >= 4) of a natural-layout work
// field with Nx a multiple of 16.  Persistent CTAs (MINB per SM: 3 at 80 registers a thread, or 2 at
// up to 128, which keeps the column-pair solve of 16 rows per lane free of spills) walk tiles of
// 16 x-slots x Nz rows
// of one y-slot, t = blockIdx.x, blockIdx.x + gridDim.x, ...  While the warps solve tile t, one
// thread's tensor copy of tile t + gridDim.x lands in a raw staging buffer (its own mbarrier, bytes
// counted), so each CTA always has its next 32 KB in flight; after the wait, the CTA moves the
// staged rows into the bank-swizzled solve tile (ZSwz16), hands the staging buffer back to the copy
// engine, solves, and stores the tile with 16-byte writes.  A copy that never lands (a bounded wait
// running out) records CANS_ERR_TIMEOUT in the plan's status word and ends the CTA.
// The register-staged float z pass (one 32-slot tile per CTA, as zpass_f32_kernel) with a tensor
// prefetch into L2: CTA b (tiles numbered row by row) first asks TMA to bring tile b + ahead into L2
// -- ahead is the number of CTAs resident at once, so that tile belongs to a CTA that starts about
// when this one ends -- and its own 16-byte loads then mostly wait for L2 instead of DRAM.  The
// prefetch has no shared-memory destination and nothing waits for it.
template <int MMAX, bool PAIR>
__global__ void __launch_bounds__(256, 3) zpass_pf_kernel(const __grid_constant__ CUtensorMap tm,
                                                          float* __restrict__ w, ZArgs a, ZTab<float> zf,
                                                          int ahead) {
  constexpr int TI = 32, NZ = 32 * MMAX, BOXZ = NZ < 256 ? NZ : 256, NBOX = NZ / BOXZ;
  constexpr bool CL = MMAX >= 4;
  const int tn = (blockIdx.y * gridDim.x + blockIdx.x) + ahead;
  if (threadIdx.x == 0 && tn < (int)(gridDim.x * gridDim.y)) {
#pragma unroll
    for (int b = 0; b < NBOX; ++b) tma_prefetch_l2_3d(&tm, (tn % gridDim.x) * TI, tn / gridDim.x, b * BOXZ);
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int rs = 32 * (MMAX + 4);
  float* sa = reinterpret_cast<float*>(smem_raw);
  float* sb = sa + rs;
  float* sc = sb + rs;
  float* tile = sc + rs;
  const int i0 = blockIdx.x * TI, j = blockIdx.y;
  const size_t plane = (size_t)a.nx * a.ny;
  float* col0 = w + (size_t)j * a.nx + i0;
  const auto Z = make_zswz<TI, MMAX>(TI, MMAX);
  stage_zrows<CL>(sa, sb, sc, zf, NZ, MMAX);
  tile_load<float>(tile, col0, plane, Z, NZ, TI, true);
  __syncthreads();
  solve_tile_f32<MMAX, PAIR>(tile, Z, a, i0, j, TI, sa, sb, sc);
  __syncthreads();
  tile_store<float>(tile, col0, plane, Z, NZ, TI, true);
}

template <int TI, int MMAX>
struct TmaSwz {
  typedef ZSwz16<MMAX> type;
};
template <int MMAX>
struct TmaSwz<32, MMAX> {
  typedef ZSwz<32, MMAX> type;
};

template <int MMAX, bool PAIR, int MINB, int TI>
__global__ void __launch_bounds__(16 * TI, MINB) zpass_tma_kernel(const __grid_constant__ CUtensorMap tm,
                                                           float* __restrict__ w, ZArgs a, ZTab<float> zf, int ntx,
                                                           int ntiles, unsigned wait_limit) {
  constexpr int NT = 16 * TI;  // 8 warps for 16-slot tiles, 16 for 32-slot tiles: one pair per warp
  constexpr int NZ = 32 * MMAX, BOXZ = NZ < 256 ? NZ : 256, NBOX = NZ / BOXZ;
  constexpr int PR = TI / 4;  // 16-byte vectors per tile row
  constexpr uint32_t TILE_BYTES = TI * NZ * 4;
  constexpr int LS = MMAX + 4;
  static_assert(MMAX >= 4 && NZ % BOXZ == 0, "full columns of 128, 256 or 512 rows");
  // every buffer at a fixed offset from the 128-byte aligned dynamic shared array (the tensor copy's
  // destination alignment), so no buffer address has to stay live in registers across the solve
  extern __shared__ __align__(128) float ztma_smem[];
  float* const stage = ztma_smem;
  float* const tile = ztma_smem + TI * NZ;
  float* const sa = tile + TI * NZ;
  float* const sb = sa + 32 * LS;
  float* const sc = sb + 32 * LS;
  uint64_t* const bar = reinterpret_cast<uint64_t*>(sc + 32 * LS);
  const int tid = threadIdx.x;
  if (tid == 0) mbar_init(bar, 1);
  stage_zrows<true>(sa, sb, sc, zf, NZ, MMAX);
  __syncthreads();
  const typename TmaSwz<TI, MMAX>::type Z = {};
  auto issue = [&](int t) {
    const int tx = t % ntx, j = t / ntx;
    mbar_arrive_expect_tx(bar, TILE_BYTES);
#pragma unroll
    for (int b = 0; b < NBOX; ++b) tma_load_3d(stage + b * BOXZ * TI, &tm, tx * TI, j, b * BOXZ, bar);
  };
  int t = blockIdx.x;
  if (tid == 0 && t < ntiles) issue(t);
  uint32_t parity = 0;
  for (; t < ntiles; t += gridDim.x) {
    const int tx = t % ntx, j = t / ntx, i0 = tx * TI;
    const bool landed = mbar_wait_bounded(bar, parity, wait_limit);
    if (__syncthreads_or(!landed)) {
      if (tid == 0) {
        atomicCAS(a.status, CANS_OK, CANS_ERR_TIMEOUT);
        mbar_wait_bounded(bar, parity, wait_limit);  // give the copy in flight a last chance to land
      }
      return;
    }
    parity ^= 1u;
    const float4* src = reinterpret_cast<const float4*>(stage);
#pragma unroll 4
    for (int e = tid; e < NZ * PR; e += NT) {
      const int k = e / PR, q = (e % PR) * 4;
      const float4 v = src[e];
      tile[Z.at(k, q)] = v.x;
      tile[Z.at(k, q + 1)] = v.y;
      tile[Z.at(k, q + 2)] = v.z;
      tile[Z.at(k, q + 3)] = v.w;
    }
    __syncthreads();
    if (tid == 0 && t + (int)gridDim.x < ntiles) {
      fence_async_smem();  // the staging reads above come before the next copy's writes
      issue(t + gridDim.x);
    }
    solve_tile_f32<MMAX, PAIR>(tile, Z, a, i0, j, TI, sa, sb, sc);
    __syncthreads();
    float* col0 = w + (size_t)j * a.nx + i0;
    const size_t plane = (size_t)a.nx * a.ny;
#pragma unroll 4
    for (int e = tid; e < NZ * PR; e += NT) {
      const int k = e / PR, q = (e % PR) * 4;
      float4 v;
      v.x = tile[Z.at(k, q)];
      v.y = tile[Z.at(k, q + 1)];
      v.z = tile[Z.at(k, q + 2)];
      v.w = tile[Z.at(k, q + 3)];
      *reinterpret_cast<float4*>(col0 + (size_t)k * plane + q) = v;
    }
    __syncthreads();
  }
}

// Two CTAs per SM for a double tile (the FP64 path: its dependent FP64 chains hide each other better,
// 1024x1024x512 FP64 solve 97.9 -> 95.1 ms, despite register spills at 128 registers), one for a float
// tile (the mixed path's marked columns: 0.22 ms against 0.25 with two).
template <typename T, int MMAX, int TIC>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 2 : 1) zpass_f64_kernel(T* __restrict__ w, ZArgs a, ZTab<double> zd, int vec,
                                                           WLay wl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int TI = TIC > 0 ? TIC : a.ti, m = a.m;
  double* sa = reinterpret_cast<double*>(smem_raw);
  double* sb = sa + 32 * m;
  double* sc = sb + 32 * m;
  T* tile = reinterpret_cast<T*>(sc + 32 * m);
  const int i0 = blockIdx.x * TI, j = blockIdx.y;
  const size_t plane = wl.zstride();
  T* col0 = w + wl.zbase(i0, j);
  const int ncols = min(TI, a.nx - i0);
  if (a.mask != nullptr) {  // skip tiles without a marked column
    bool any = false;
    for (int c = 0; c < ncols; ++c) any |= a.mask[(size_t)j * a.nx + i0 + c] != 0;
    if (!any) return;
  }
  const auto Z = make_zswz<TIC, MMAX>(TI, m);
  stage_zrows<false>(sa, sb, sc, zd, a.nz, m);
  tile_load<T>(tile, col0, plane, Z, a.nz, ncols, vec != 0);
  __syncthreads();
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const double muy = a.muy_d[j] + a.shift;
  auto marked = [&](int i) { return a.mask == nullptr || a.mask[(size_t)j * a.nx + i]; };
  auto single = [&](int cidx) {
    const int i = i0 + cidx;
    if (!marked(i)) return;
    const double mu = a.mux_d[i] + muy;
    if (a.singular && i == 0 && j == 0) {
      const double target = (a.gauge != nullptr) ? a.gauge_scale * (*a.gauge) : 0.0;
      zsolve_column<MMAX, double, T, true>(tile, cidx, Z, a.nz, mu, sa, sb, sc, a.dzf, target, a.compat);
    } else {
      zsolve_column<MMAX, double, T, false>(tile, cidx, Z, a.nz, mu, sa, sb, sc, nullptr, 0.0);
    }
  };
  if (MMAX >= 2 && a.xpairs) {  // x periodic: slots 2q, 2q+1 (q >= 1) share their shift, one factorisation
    for (int q = warp; 2 * q < ncols; q += nwarps) {
      const int c0 = 2 * q, i = i0 + c0;
      if (i == 0 || !marked(i) || !marked(i + 1)) {
        single(c0);
        single(c0 + 1);
      } else if constexpr (MMAX >= 2) {
        zsolve_pair<MMAX, double, T, decltype(Z), false, false>(tile, c0, c0 + 1, Z, a.nz, a.mux_d[i] + muy, sa, sb,
                                                                 sc);
      }
    }
  } else {
    for (int cidx = warp; cidx < ncols; cidx += nwarps) single(cidx);
  }
  __syncthreads();
  tile_store<T>(tile, col0, plane, Z, a.nz, ncols, vec != 0);
}

static ZArgs zargs(const cans_plan_s* P, int ti, const double* gauge, double* compat) {
  ZArgs a;
  a.compat = compat;
  a.status = P->status_d;
  a.nx = P->n[0];
  a.ny = P->n[1];
  a.nz = P->n[2];
  a.ti = ti;
  a.m = P->z_m;
  a.singular = P->singular ? 1 : 0;
  a.shift = P->shift;
  a.mask = nullptr;
  a.mux_d = P->mux_d;
  a.muy_d = P->muy_d;
  a.mux_f = P->mux_f;
  a.muy_f = P->muy_f;
  a.dzf = P->dzf_d;
  a.gauge = gauge;
  a.gauge_scale = P->gauge_scale;
  a.i_end = P->n[0];
  a.j_end = P->n[1];
  // periodic x: slots 2q, 2q+1 hold one wavenumber's Re / Im parts (equal shift); tiles of an even
  // width hold whole pairs
  a.xpairs = (P->bc[0] == BC_P && P->n[0] % 2 == 0 && ti % 2 == 0) ? 1 : 0;
  return a;
}

// ---- TMA-fed float z pass: host side ----------------------------------------------------------
// The tensor-map encoder is a driver function; the runtime hands out its address, so the library
// needs no link against the driver library.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(ptr);
  });
  return fn;
}

// Shapes the TMA kernel takes: float natural-layout work field, Nx a multiple of 16 (16-slot tiles,
// 64-byte box rows), full columns of 128, 256 or 512 rows, a 16-byte aligned field.
bool ztma_feasible(const cans_plan_s* P, const void* w) {
  return !P->wblk && P->n[0] % 16 == 0 && P->z_mmax >= 4 && P->n[2] == 32 * P->z_mmax &&
         (reinterpret_cast<uintptr_t>(w) & 15) == 0 && encode_tiled() != nullptr;
}

constexpr unsigned kTmaWaitLimit = 1u << 20;  // polls of one copy's barrier (~0.3 s) before a timeout

template <int MMAX, int MINB, int TI>
static cudaError_t ztma_m(const cans_plan_s* P, float* w, cudaStream_t st) {
  constexpr int NZ = 32 * MMAX;
  const int nx = P->n[0], ny = P->n[1];
  CUtensorMap tm;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)NZ};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4};
  const cuuint32_t box[3] = {TI, 1, (cuuint32_t)(NZ < 256 ? NZ : 256)};
  const cuuint32_t estr[3] = {1, 1, 1};
  // box rows are 64 bytes: no promotion to 128-byte L2 lines (their other half belongs to the
  // neighbouring tile, which another CTA reads at another time)
  CUtensorMapL2promotion prom = CU_TENSOR_MAP_L2_PROMOTION_NONE;
  if (const char* ev = std::getenv("CANS_Z_TMA_L2")) prom = ev[0] == '1' ? CU_TENSOR_MAP_L2_PROMOTION_L2_128B
                                                       : (ev[0] == '6' ? CU_TENSOR_MAP_L2_PROMOTION_L2_64B : prom);
  if (encode_tiled()(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, w, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, prom,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  ZArgs a = zargs(P, TI, nullptr, nullptr);
  a.mask = P->mask_d;
  const bool pair = P->bc[0] == BC_P;  // Nx is even: every 16-slot tile holds whole Re / Im pairs
  auto kern = pair ? zpass_tma_kernel<MMAX, true, MINB, TI> : zpass_tma_kernel<MMAX, false, MINB, TI>;
  const size_t smem = 2 * (size_t)TI * NZ * 4 + 3 * 32 * (MMAX + 4) * 4 + 16;
  cudaError_t e = set_smem((const void*)kern, smem);
  if (e != cudaSuccess) return e;
  // persistent grid: every resident CTA slot of the device (cached per device and kernel)
  static std::mutex lock;
  static int cached[16][2] = {};  // per device and pair flag, for this instantiation
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  int per_sm = 0, sms = 0;
  {
    std::lock_guard<std::mutex> g(lock);
    int& c = cached[dev & 15][pair ? 1 : 0];
    if (c == 0) {
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, kern, 16 * TI, smem)) != cudaSuccess) return e;
      c = c < 1 ? 1 : c;
    }
    per_sm = c;
  }
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int ntx = nx / TI, ntiles = ntx * ny;
  const int grid = ntiles < per_sm * sms ? ntiles : per_sm * sms;
  kern<<<grid, 16 * TI, smem, st>>>(tm, w, a, P->zt_f, ntx, ntiles, kTmaWaitLimit);
  return cudaGetLastError();
}

// shape variants: 1 = one 512-thread CTA per SM on 32-slot tiles (128-byte rows), 2 / 3 = two or
// three 256-thread CTAs per SM on 16-slot tiles
template <int MMAX>
static cudaError_t zpf_m(const cans_plan_s* P, float* w, cudaStream_t st) {
  constexpr int TI = 32, NZ = 32 * MMAX;
  const int nx = P->n[0], ny = P->n[1];
  CUtensorMap tm;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)NZ};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4};
  const cuuint32_t box[3] = {TI, 1, (cuuint32_t)(NZ < 256 ? NZ : 256)};
  const cuuint32_t estr[3] = {1, 1, 1};
  if (encode_tiled()(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, w, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  ZArgs a = zargs(P, TI, nullptr, nullptr);
  a.mask = P->mask_d;
  const bool pair = P->bc[0] == BC_P;
  auto kern = pair ? zpass_pf_kernel<MMAX, true> : zpass_pf_kernel<MMAX, false>;
  const size_t smem = 3 * 32 * (MMAX + 4) * 4 + (size_t)TI * NZ * 4;
  cudaError_t e = set_smem((const void*)kern, smem);
  if (e != cudaSuccess) return e;
  static std::mutex lock;
  static int cached[16][2] = {};
  int dev = 0, per_sm = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> g(lock);
    int& c = cached[dev & 15][pair ? 1 : 0];
    if (c == 0) {
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, kern, 256, smem)) != cudaSuccess) return e;
      c = c < 1 ? 1 : c;
    }
    per_sm = c;
  }
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  dim3 grid(nx / TI, ny);
  kern<<<grid, 256, smem, st>>>(tm, w, a, P->zt_f, per_sm * sms);
  return cudaGetLastError();
}

template <int MMAX>
static cudaError_t ztma_v(const cans_plan_s* P, float* w, cudaStream_t st) {
  if (P->z_tma_ctas == 4 && P->n[0] % 32 == 0) return zpf_m<MMAX>(P, w, st);
  if (P->z_tma_ctas == 1 && P->n[0] % 32 == 0) return ztma_m<MMAX, 1, 32>(P, w, st);
  if (P->z_tma_ctas == 3) return ztma_m<MMAX, 3, 16>(P, w, st);
  return ztma_m<MMAX, 2, 16>(P, w, st);
}

static cudaError_t launch_ztma(const cans_plan_s* P, float* w, cudaStream_t st) {
  switch (P->z_mmax) {
    case 4: return ztma_v<4>(P, w, st);
    case 8: return ztma_v<8>(P, w, st);
    default: return ztma_v<16>(P, w, st);
  }
}

// part: -1 both kernels, 0 the float columns only, 1 the marked double columns only (mixed path)
template <typename T, int MMAX, int TIC>
static cudaError_t z_mt(const cans_plan_s* P, T* w, const double* gauge, cudaStream_t st, int part,
                        double* compat) {
  const WLay wl = wlay(P, sizeof(T) == 4);
  const int vec = ((wl.blk || P->n[0] % 4 == 0) && (reinterpret_cast<uintptr_t>(w) & 15) == 0) ? 1 : 0;
  if (sizeof(T) == 4) {
    // float columns first, then the double columns of the marked bounding box
    cudaError_t e = cudaSuccess;
    const bool tma = MMAX >= 4 && P->z_tma && ztma_feasible(P, w);
    const bool p2 = !tma && MMAX >= 4 && TIC == 32 && P->z_p2 && P->n[2] == 32 * MMAX && P->n[0] % 32 == 0 &&
                    !wl.blk && (reinterpret_cast<uintptr_t>(w) & 15) == 0;
    // short columns on the staged kernel of a tiny field: the marked columns are solved in FP64 inside it,
    // one launch fewer per z pass on a latency-bound chain (32^3 mixed with 2 sweeps: 139 -> 130 us); on
    // larger fields the separate double kernel overlaps better with other work (64-problem ensemble
    // 4.63 ms separate, 4.70 fused), so z_fuse64 = 1 fuses up to 2^16 points only, 2 always
    const size_t npts = (size_t)P->n[0] * P->n[1] * P->n[2];
    const bool fuse = !tma && !p2 && P->z_tma != 2 && MMAX <= 4 && P->mask_d != nullptr &&
                      (P->z_fuse64 == 2 || (P->z_fuse64 == 1 && npts <= ((size_t)1 << 16)));
    if (part != 1) {
      if (tma) {
        e = launch_ztma(P, reinterpret_cast<float*>(w), st);
      } else if (P->z_tma == 2) {
        return cudaErrorNotSupported;  // the TMA kernel was required and cannot take this shape
      } else if (p2) {
        // pair-granular tiles fetched by cp.async (full columns, whole 32-slot tiles; the column pairs of
        // a periodic x share their factorisation)
        if constexpr (MMAX >= 4) {
          ZArgs a = zargs(P, 32, gauge, nullptr);
          a.mask = P->mask_d;
          const size_t smem = 3 * 32 * (MMAX + 4) * sizeof(float) + (size_t)32 * 32 * MMAX * sizeof(float);
          auto kern = P->bc[0] == BC_P ? zpass_p2_kernel<MMAX, true> : zpass_p2_kernel<MMAX, false>;
          e = set_smem((const void*)kern, smem);
          if (e != cudaSuccess) return e;
          kern<<<dim3(P->n[0] / 32, P->n[1]), 256, smem, st>>>(reinterpret_cast<float*>(w), a, P->zt_f, wl);
          e = cudaGetLastError();
        }
      } else {
        ZArgs a = zargs(P, P->z_ti[1], gauge, fuse ? compat : nullptr);
        a.mask = P->mask_d;
        const size_t smem = 3 * 32 * (a.m + 4) * sizeof(float) + P->z_smem[1] +
                            (fuse ? 3 * 32 * (size_t)a.m * sizeof(double) + sizeof(double) : 0);
        dim3 grid((a.nx + a.ti - 1) / a.ti, a.ny);
        // pairs of equal eigenvalues: periodic x, every tile an even number of whole pairs
        const bool pair = MMAX >= 4 && P->bc[0] == BC_P && a.nx % 2 == 0 && a.ti % 2 == 0;
        constexpr bool F64 = MMAX <= 4;  // the fused variant exists for short columns only
        auto kern = pair ? (fuse ? zpass_f32_kernel<MMAX, TIC, (MMAX >= 4), F64> : zpass_f32_kernel<MMAX, TIC, (MMAX >= 4)>)
                         : (fuse ? zpass_f32_kernel<MMAX, TIC, false, F64> : zpass_f32_kernel<MMAX, TIC, false>);
        e = set_smem((const void*)kern, smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, 256, smem, st>>>(reinterpret_cast<float*>(w), a, P->zt_f, vec, wl, P->zt_d);
        e = cudaGetLastError();
      }
      if (e != cudaSuccess || part == 0) return e;
    }
    if (fuse) return cudaSuccess;  // the marked columns were solved with the float ones
    ZArgs b = zargs(P, P->z_ti[1], gauge, compat);
    b.mask = P->mask_d;
    const size_t smem64 = 3 * 32 * b.m * sizeof(double) + P->z_smem[1];
    e = set_smem((const void*)zpass_f64_kernel<T, MMAX, TIC>, smem64);
    if (e != cudaSuccess) return e;
    dim3 grid64((P->mask_i_end + b.ti - 1) / b.ti, P->mask_j_end);
    if (grid64.x > 0 && grid64.y > 0) zpass_f64_kernel<T, MMAX, TIC><<<grid64, 256, smem64, st>>>(w, b, P->zt_d, vec, wl);
    return cudaGetLastError();
  }
  ZArgs a = zargs(P, P->z_ti[0], gauge, compat);
  const size_t smem = 3 * 32 * a.m * sizeof(double) + P->z_smem[0];
  cudaError_t e = set_smem((const void*)zpass_f64_kernel<T, MMAX, TIC>, smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.nx + a.ti - 1) / a.ti, a.ny);
  zpass_f64_kernel<T, MMAX, TIC><<<grid, 256, smem, st>>>(w, a, P->zt_d, vec, wl);
  return cudaGetLastError();
}

// compile-time tile widths for the common shapes (the z tile is TI x-slots wide, a power of two)
template <typename T, int MMAX>
static cudaError_t z_m(const cans_plan_s* P, T* w, const double* gauge, cudaStream_t st, int part, double* compat) {
  switch (P->z_ti[sizeof(T) == 4 ? 1 : 0]) {
    case 32: return z_mt<T, MMAX, 32>(P, w, gauge, st, part, compat);
    case 16: return z_mt<T, MMAX, 16>(P, w, gauge, st, part, compat);
    case 8: return z_mt<T, MMAX, 8>(P, w, gauge, st, part, compat);
    default: return z_mt<T, MMAX, 0>(P, w, gauge, st, part, compat);
  }
}

template <typename T>
cudaError_t launch_z(const cans_plan_s* P, T* w, const double* gauge, cudaStream_t st, int part, double* compat) {
  if (P->bc[2] == BC_P) return (part == 1) ? cudaSuccess : launch_zspec<T>(P, w, gauge, st, compat);
  switch (P->z_mmax) {
    case 1: return z_m<T, 1>(P, w, gauge, st, part, compat);
    case 2: return z_m<T, 2>(P, w, gauge, st, part, compat);
    case 4: return z_m<T, 4>(P, w, gauge, st, part, compat);
    case 8: return z_m<T, 8>(P, w, gauge, st, part, compat);
    default: return z_m<T, 16>(P, w, gauge, st, part, compat);
  }
}

template cudaError_t launch_z<double>(const cans_plan_s*, double*, const double*, cudaStream_t, int, double*);
template cudaError_t launch_z<float>(const cans_plan_s*, float*, const double*, cudaStream_t, int, double*);

}  // namespace cans
