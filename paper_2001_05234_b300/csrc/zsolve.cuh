// Tridiagonal solves along z, one per (x, y) mode (Eq. poi_reduced; Gauss elimination along a
// non-uniform z grid).
//
// A CTA stages a tile of TI consecutive x-slots x Nz rows (one y-slot) in shared memory with
// coalesced loads, then one warp solves one column at a time: lane p owns the contiguous rows
// [p*m, p*m + m) (m = ceil(Nz/32)).  Each lane eliminates its own rows, expressing them through the
// last unknown of the previous lane's segment and of its own segment (a partitioned Thomas
// solve); the 32 interface unknowns form a tridiagonal system that the warp solves by parallel
// cyclic reduction over shuffles; each lane then back-substitutes its rows.  Rows past Nz are
// identity rows.  The column's precision C (float or double) is independent of the storage type.
#pragma once
#include <cuda_runtime.h>

#include "dfloat.cuh"

namespace cans {

template <typename T>
struct ZTab {
  const T* a;  // sub-diagonal a_k (a_0 = 0 at a wall)
  const T* b;  // diagonal b_k (without mu)
  const T* c;  // super-diagonal c_k (c_{Nz-1} = 0 at a wall)
};

// Reciprocal: approximate (one MUFU op, ~1 ulp) for float columns -- the mixed path corrects the
// float solve by refinement anyway.  Double columns (below) take the approximate reciprocal refined
// by two Newton steps: within about 1 ulp, not correctly rounded.
__device__ __forceinline__ float rcp_(float x) {
  float r;
  asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// 1/x in double: the hardware's approximate reciprocal refined by two Newton steps
// y <- y + y (1 - x y), each squaring the relative error; the pivots of the z systems are normal,
// nonzero numbers (diagonal dominance), so the flush-to-zero approximation is safe here.
__device__ __forceinline__ double rcp_(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}

// Swizzled position of (row k, column i) inside the [Nz][TI] tile.  Every lane owns m = 2^sh rows
// (rows past Nz are identity rows), so row k belongs to lane seg = k >> sh; the column index is
// xor-ed with seg (the 32 lanes reading one column hit 32 banks) and, when m >= 4, with k & 3 (the
// row-major copy phases, four rows at a time, spread over all banks as well).
// TI_ > 0 fixes the tile width at compile time (with M_ the rows per lane), so that every index
// folds into per-lane constants; TI_ = 0 keeps both at run time.
template <int TI_ = 0, int M_ = 0>
struct ZSwz {
  int TI, sh, low;
  __device__ __forceinline__ int ti() const { return TI_ > 0 ? TI_ : TI; }
  __device__ __forceinline__ int shift() const { return TI_ > 0 ? ilog2_c(M_) : sh; }
  __device__ __forceinline__ int lowm() const { return TI_ > 0 ? (M_ >= 4 ? 3 : 0) : low; }
  __device__ __forceinline__ int seg(int k) const { return k >> shift(); }
  __device__ __forceinline__ int at(int k, int i, int sg) const {
    return k * ti() + (i ^ ((sg ^ (k & lowm())) & (ti() - 1)));
  }
  __device__ __forceinline__ int at(int k, int i) const { return at(k, i, seg(k)); }
  static __host__ __device__ constexpr int ilog2_c(int x) { return x <= 1 ? 0 : 1 + ilog2_c(x / 2); }
};
// 16-wide tiles (the TMA-fed z pass): rows k and k+1 (k even) share one 32-word line, so the XOR
// pattern spans all 32 banks -- a dense 16-word row alone could reach only 16.  Lanes reading one
// column (rows lane*M + r) and the row-major copy phases (8 rows x 4 vectors per warp) both hit 32
// distinct banks for M = 4, 8, 16 (checked by enumeration).
template <int M_>
struct ZSwz16 {
  static constexpr int SH = M_ >= 16 ? 4 : (M_ >= 8 ? 3 : (M_ >= 4 ? 2 : (M_ >= 2 ? 1 : 0)));
  __device__ __forceinline__ int ti() const { return 16; }
  __device__ __forceinline__ int at(int k, int i, int sg) const {
    return ((k >> 1) << 5) + ((((k & 1) << 4) | i) ^ ((sg ^ ((k >> 1) & 3)) & 31));
  }
  __device__ __forceinline__ int at(int k, int i) const { return at(k, i, k >> SH); }
};

// Pair-granular 32-wide tiles (the column pairs 2p, 2p+1 of a periodic x direction stay adjacent: one
// 8-byte word per row and pair).  The pair index is XOR-ed with the low four bits of the owning lane's
// segment and with k & 3, so the 16 lanes of each half-warp's 8-byte accesses of one pair reach 16
// distinct bank pairs; a 4-byte access of one column from all 32 lanes meets 2-way conflicts (lanes l
// and l + 16).  M_ rows per lane (a power of two).
template <int M_>
struct ZSwzP {
  static constexpr int SH = ZSwz<>::ilog2_c(M_);
  __device__ __forceinline__ int ti() const { return 32; }
  __device__ __forceinline__ int at(int k, int i, int sg) const {
    return k * 32 + ((((i >> 1) ^ ((sg ^ (k & 3)) & 15)) << 1) | (i & 1));
  }
  __device__ __forceinline__ int at(int k, int i) const { return at(k, i, k >> SH); }
};

template <int TI_ = 0, int M_ = 0>
__device__ __forceinline__ ZSwz<TI_, M_> make_zswz(int TI, int m) {
  ZSwz<TI_, M_> s;
  s.TI = TI;
  s.sh = 0;
  while ((1 << s.sh) < m) ++s.sh;
  s.low = (m >= 4) ? 3 : 0;
  return s;
}

// Per-CTA copy of the z rows.  Row k = lane*m + r of a lane's segment sits at [r*32 + lane] (the 32
// lanes of a warp read 32 consecutive words), or, with CL (float rows, m >= 4), at
// [lane*(m+4) + r]: each lane's rows are contiguous, so four rows come in one 16-byte load, and the
// padded lane stride keeps every quarter-warp's 16-byte loads on distinct banks.  Rows past Nz become
// identity rows (a = c = 0, b = 1).
template <bool CL = false, typename C, typename S>
__device__ __forceinline__ void stage_zrows(C* sa, C* sb, C* sc, const ZTab<S>& zt, int Nz, int m) {
  for (int q = threadIdx.x; q < 32 * m; q += blockDim.x) {
    const int lane = q & 31, r = q >> 5;
    const int k = lane * m + r;
    const bool in = k < Nz;
    const int at = CL ? lane * (m + 4) + r : q;
    sa[at] = in ? (C)zt.a[k] : (C)0;
    sb[at] = in ? (C)zt.b[k] : (C)1;
    sc[at] = in ? (C)zt.c[k] : (C)0;
  }
}

__device__ __forceinline__ float f4_get(const float4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// Solve one column (tile column `col`) in precision C with rows staged by stage_zrows.  FULL: the
// caller guarantees Nz = 32 MMAX (no identity rows), which removes every row-validity test.
// mu is the x-y eigenvalue term of the mode.  SING: the singular Neumann mode -- the right-hand side
// is first projected on the compatible subspace (sum_k dzf_k d_k = 0), the last row is replaced by
// x = 0, and the result is shifted to the dzf-weighted mean `target`; the removed part
// sum_k dzf_k d_k goes to *compat when compat is not NULL (the compatibility check of the status word).
template <int MMAX, typename C, typename T, bool SING, typename ZS, bool FULL = false, bool CL = false>
__device__ __forceinline__ void zsolve_column(T* tile, int col, const ZS& Z, int Nz, C mu, const C* sa,
                                              const C* sb, const C* sc, const double* weights, C target,
                                              double* compat = nullptr) {
  const int lane = threadIdx.x & 31;
  constexpr int m = MMAX;  // rows per lane (compile time: keeps the row arrays in registers)
  static_assert(!CL || (MMAX >= 4 && sizeof(C) == 4), "lane-contiguous rows: float, four rows per load");
  constexpr int LS = MMAX + 4;
  float4 A4, B4, C4;  // CL: rows r .. r+3 of this lane's coefficients
  auto coefs = [&](int r, C& a, C& b, C& c) {
    if constexpr (CL) {
      if ((r & 3) == 0) {
        A4 = *reinterpret_cast<const float4*>(sa + lane * LS + r);
        B4 = *reinterpret_cast<const float4*>(sb + lane * LS + r);
        C4 = *reinterpret_cast<const float4*>(sc + lane * LS + r);
      }
      a = f4_get(A4, r & 3);
      b = f4_get(B4, r & 3);
      c = f4_get(C4, r & 3);
    } else {
      a = sa[r * 32 + lane];
      b = sb[r * 32 + lane];
      c = sc[r * 32 + lane];
    }
  };
  const int k0 = lane * m;
  const unsigned full = 0xffffffffu;
  C proj = 0;
  if (SING) {
    C sw = 0, swd = 0;
    for (int r = 0; r < m; ++r) {
      const int k = k0 + r;
      if (FULL || k < Nz) {
        const C w = (C)weights[k];
        sw += w;
        swd += w * cvt<C>(tile[Z.at(k, col, lane)]);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sw += __shfl_xor_sync(full, sw, o);
      swd += __shfl_xor_sync(full, swd, o);
    }
    proj = swd / sw;
    if (compat != nullptr && lane == 0) *compat = (double)swd;
  }
  C cp[MMAX], dp[MMAX], lp[MMAX];
  C rr = 0;
  // local forward elimination over rows r = 0..m-2 of the segment
  C cprev = 0, dprev = 0, lprev = 0;
#pragma unroll
  for (int r = 0; r < MMAX; ++r) {
    if (r < m - 1) {
      const int k = k0 + r;
      // identity rows past Nz keep b = 1 (with mu added, 1 + mu could vanish)
      C a, b, c, d = 0;
      coefs(r, a, b, c);
      b += (FULL || k < Nz) ? mu : (C)0;
      if (FULL || k < Nz) d = cvt<C>(tile[Z.at(k, col, lane)]) - proj;
      if (SING && k == Nz - 1) {
        a = 0;
        b = 1;
        c = 0;
        d = 0;
      }
      const C inv = rcp_(b - a * cprev);
      const bool last_inner = (r == m - 2);
      cp[r] = last_inner ? (C)0 : c * inv;
      if (last_inner) rr = -c * inv;
      dp[r] = (d - a * dprev) * inv;
      lp[r] = ((r == 0) ? -a : -a * lprev) * inv;
      cprev = c * inv;
      dprev = dp[r];
      lprev = lp[r];
    }
  }
  // backward sweep for the expressions x_r = D + V E_prev + W E_own at r = m-2 and r = 0
  C Dl = 0, Vl = 1, Wl = 0, Df = 0, Vf = 0, Wf = 1;
  if (m >= 2) {
    C D = 0, V = 0, W = 0;
#pragma unroll
    for (int r = MMAX - 1; r >= 0; --r) {
      if (r <= m - 2) {
        if (r == m - 2) {
          D = dp[r];
          V = lp[r];
          W = rr;
          Dl = D;
          Vl = V;
          Wl = W;
        } else {
          D = dp[r] - cp[r] * D;
          V = lp[r] - cp[r] * V;
          W = -cp[r] * W;
        }
      }
    }
    Df = D;
    Vf = V;
    Wf = W;
  }
  // this segment's last row ties the interface unknowns together
  const int kl = k0 + m - 1;
  const int rl = m - 1;
  C al, bl, cl, dl = 0;
  if (CL && ((m - 1) & 3) != 0) {  // the last row's group of four was loaded by the forward loop
    al = f4_get(A4, rl & 3);
    bl = f4_get(B4, rl & 3);
    cl = f4_get(C4, rl & 3);
  } else {
    coefs(rl, al, bl, cl);
  }
  bl += (FULL || kl < Nz) ? mu : (C)0;
  if (FULL || kl < Nz) dl = cvt<C>(tile[Z.at(kl, col, lane)]) - proj;
  if (SING && kl == Nz - 1) {
    al = 0;
    bl = 1;
    cl = 0;
    dl = 0;
  }
  const C Dfn = __shfl_down_sync(full, Df, 1);
  const C Vfn = __shfl_down_sync(full, Vf, 1);
  const C Wfn = __shfl_down_sync(full, Wf, 1);
  C alpha = (lane == 0) ? (C)0 : al * Vl;
  C beta = bl + al * Wl + ((lane < 31) ? cl * Vfn : (C)0);
  C gamma = (lane < 31) ? cl * Wfn : (C)0;
  C delta = dl - al * Dl - ((lane < 31) ? cl * Dfn : (C)0);
  // parallel cyclic reduction of the 32 interface equations
#pragma unroll
  for (int s = 1; s < 32; s <<= 1) {
    C am = __shfl_up_sync(full, alpha, s), bm = __shfl_up_sync(full, beta, s);
    C gm = __shfl_up_sync(full, gamma, s), dm = __shfl_up_sync(full, delta, s);
    C ap = __shfl_down_sync(full, alpha, s), bp = __shfl_down_sync(full, beta, s);
    C gp = __shfl_down_sync(full, gamma, s), dpv = __shfl_down_sync(full, delta, s);
    if (lane < s) { am = 0; bm = 1; gm = 0; dm = 0; }
    if (lane + s > 31) { ap = 0; bp = 1; gp = 0; dpv = 0; }
    const C k1 = alpha * rcp_(bm), k2 = gamma * rcp_(bp);
    const C na = -am * k1, ng = -gp * k2;
    const C nb = beta - gm * k1 - ap * k2;
    const C nd = delta - dm * k1 - dpv * k2;
    alpha = na;
    beta = nb;
    gamma = ng;
    delta = nd;
  }
  const C E = delta * rcp_(beta);
  C Ep = __shfl_up_sync(full, E, 1);
  if (lane == 0) Ep = 0;
  // back-substitution, written straight into the tile
  if (FULL || lane * m + m - 1 < Nz) tile[Z.at(k0 + m - 1, col, lane)] = cvt<T>(E);
  C xn = E;
#pragma unroll
  for (int r = MMAX - 1; r >= 0; --r) {
    if (r <= m - 2) {
      if (r == m - 2)
        xn = dp[r] + lp[r] * Ep + rr * E;
      else
        xn = dp[r] + lp[r] * Ep - cp[r] * xn;
      if (FULL || k0 + r < Nz) tile[Z.at(k0 + r, col, lane)] = cvt<T>(xn);
    }
  }
  if (SING) {
    // shift the column to the weighted mean `target`
    C sw = 0, swx = 0;
    for (int r = 0; r < m; ++r) {
      const int k = k0 + r;
      if (FULL || k < Nz) {
        const C w = (C)weights[k];
        sw += w;
        swx += w * cvt<C>(tile[Z.at(k, col, lane)]);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sw += __shfl_xor_sync(full, sw, o);
      swx += __shfl_xor_sync(full, swx, o);
    }
    const C shift = swx / sw - target;
    for (int r = 0; r < m; ++r) {
      const int k = k0 + r;
      if (FULL || k < Nz) tile[Z.at(k, col, lane)] = cvt<T>(cvt<C>(tile[Z.at(k, col, lane)]) - shift);
    }
  }
}


// Two columns with the same shift mu (the Re and Im slots of one periodic x wavenumber): the
// coefficient-only parts of the partitioned solve above (pivots, spikes, the reduced system's
// matrix and its cyclic reduction) are computed once and applied to both right-hand sides.
// Non-singular columns; compute type C, storage type T.  When C is T, the second column's forward
// values go back into its own tile rows instead of registers (register budget of the float kernel).
template <int MMAX, typename C, typename T, typename ZS, bool FULL, bool CL>
__device__ __forceinline__ void zsolve_pair(T* tile, int col0, int col1, const ZS& Z, int Nz, C mu, const C* sa,
                                            const C* sb, const C* sc) {
  constexpr bool IN_TILE = sizeof(C) == sizeof(T);
  const int lane = threadIdx.x & 31;
  constexpr int m = MMAX;
  static_assert(MMAX >= 2, "two or more rows per lane");
  static_assert(!CL || (MMAX >= 4 && sizeof(C) == 4), "lane-contiguous rows: float, four rows per load");
  constexpr int LS = MMAX + 4;
  float4 A4, B4, C4;
  auto coefs = [&](int r, C& a, C& b, C& c) {
    if constexpr (CL) {
      if ((r & 3) == 0) {
        A4 = *reinterpret_cast<const float4*>(sa + lane * LS + r);
        B4 = *reinterpret_cast<const float4*>(sb + lane * LS + r);
        C4 = *reinterpret_cast<const float4*>(sc + lane * LS + r);
      }
      a = f4_get(A4, r & 3);
      b = f4_get(B4, r & 3);
      c = f4_get(C4, r & 3);
    } else {
      a = sa[r * 32 + lane];
      b = sb[r * 32 + lane];
      c = sc[r * 32 + lane];
    }
  };
  const int k0 = lane * m;
  const unsigned full = 0xffffffffu;
  C cp[MMAX], lp[MMAX], dp0[MMAX], dp1[IN_TILE ? 1 : MMAX];
  C rr = 0, cprev = 0, lprev = 0, d0prev = 0, d1prev = 0;
  auto t1 = [&](int k) -> T& { return tile[Z.at(k, col1, lane)]; };
  auto put1 = [&](int r, int k, C v) {
    if constexpr (IN_TILE) {
      if (FULL || k < Nz) t1(k) = (T)v;
    } else {
      dp1[r] = v;
    }
  };
  auto get1 = [&](int r, int k) -> C {
    if constexpr (IN_TILE)
      return (FULL || k < Nz) ? (C)t1(k) : (C)0;
    else
      return dp1[r];
  };
#pragma unroll
  for (int r = 0; r < m - 1; ++r) {
    const int k = k0 + r;
    C a, b, c, d0 = 0, d1 = 0;
    coefs(r, a, b, c);
    b += (FULL || k < Nz) ? mu : (C)0;
    if (FULL || k < Nz) {
      d0 = cvt<C>(tile[Z.at(k, col0, lane)]);
      d1 = cvt<C>(t1(k));
    }
    const C inv = rcp_(b - a * cprev);
    const bool last_inner = (r == m - 2);
    cp[r] = last_inner ? (C)0 : c * inv;
    if (last_inner) rr = -c * inv;
    dp0[r] = (d0 - a * d0prev) * inv;
    const C dp1r = (d1 - a * d1prev) * inv;
    put1(r, k, dp1r);
    lp[r] = ((r == 0) ? -a : -a * lprev) * inv;
    cprev = c * inv;
    d0prev = dp0[r];
    d1prev = dp1r;
    lprev = lp[r];
  }
  C Dl0, Dl1, Vl, Wl, Df0, Df1, Vf, Wf;
  {
    C D0 = 0, D1 = 0, V = 0, W = 0;
#pragma unroll
    for (int r = m - 2; r >= 0; --r) {
      const C dp1r = get1(r, k0 + r);
      if (r == m - 2) {
        D0 = dp0[r];
        D1 = dp1r;
        V = lp[r];
        W = rr;
        Dl0 = D0;
        Dl1 = D1;
        Vl = V;
        Wl = W;
      } else {
        D0 = dp0[r] - cp[r] * D0;
        D1 = dp1r - cp[r] * D1;
        V = lp[r] - cp[r] * V;
        W = -cp[r] * W;
      }
    }
    Df0 = D0;
    Df1 = D1;
    Vf = V;
    Wf = W;
  }
  const int kl = k0 + m - 1;
  const int rl = m - 1;
  C al, bl, cl, dl0 = 0, dl1 = 0;
  if (CL && ((m - 1) & 3) != 0) {  // the last row's group of four was loaded by the forward loop
    al = f4_get(A4, rl & 3);
    bl = f4_get(B4, rl & 3);
    cl = f4_get(C4, rl & 3);
  } else {
    coefs(rl, al, bl, cl);
  }
  bl += (FULL || kl < Nz) ? mu : (C)0;
  if (FULL || kl < Nz) {
    dl0 = cvt<C>(tile[Z.at(kl, col0, lane)]);
    dl1 = cvt<C>(t1(kl));
  }
  const C Dfn0 = __shfl_down_sync(full, Df0, 1);
  const C Dfn1 = __shfl_down_sync(full, Df1, 1);
  const C Vfn = __shfl_down_sync(full, Vf, 1);
  const C Wfn = __shfl_down_sync(full, Wf, 1);
  const bool hasn = lane < 31;
  C alpha = (lane == 0) ? (C)0 : al * Vl;
  C beta = bl + al * Wl + (hasn ? cl * Vfn : (C)0);
  C gamma = hasn ? cl * Wfn : (C)0;
  C delta0 = dl0 - al * Dl0 - (hasn ? cl * Dfn0 : (C)0);
  C delta1 = dl1 - al * Dl1 - (hasn ? cl * Dfn1 : (C)0);
#pragma unroll
  for (int s = 1; s < 32; s <<= 1) {
    C am = __shfl_up_sync(full, alpha, s), bm = __shfl_up_sync(full, beta, s);
    C gm = __shfl_up_sync(full, gamma, s);
    C dm0 = __shfl_up_sync(full, delta0, s), dm1 = __shfl_up_sync(full, delta1, s);
    C ap = __shfl_down_sync(full, alpha, s), bp = __shfl_down_sync(full, beta, s);
    C gp = __shfl_down_sync(full, gamma, s);
    C dq0 = __shfl_down_sync(full, delta0, s), dq1 = __shfl_down_sync(full, delta1, s);
    if (lane < s) {
      am = 0;
      bm = 1;
      gm = 0;
      dm0 = 0;
      dm1 = 0;
    }
    if (lane + s > 31) {
      ap = 0;
      bp = 1;
      gp = 0;
      dq0 = 0;
      dq1 = 0;
    }
    const C k1 = alpha * rcp_(bm), k2 = gamma * rcp_(bp);
    const C na = -am * k1, ng = -gp * k2;
    const C nb = beta - gm * k1 - ap * k2;
    delta0 = delta0 - dm0 * k1 - dq0 * k2;
    delta1 = delta1 - dm1 * k1 - dq1 * k2;
    alpha = na;
    beta = nb;
    gamma = ng;
  }
  const C ib = rcp_(beta);
  const C E0 = delta0 * ib, E1 = delta1 * ib;
  C Ep0 = __shfl_up_sync(full, E0, 1), Ep1 = __shfl_up_sync(full, E1, 1);
  if (lane == 0) {
    Ep0 = 0;
    Ep1 = 0;
  }
  if (FULL || kl < Nz) {
    tile[Z.at(kl, col0, lane)] = cvt<T>(E0);
    t1(kl) = cvt<T>(E1);
  }
  C x0 = E0, x1 = E1;
#pragma unroll
  for (int r = m - 2; r >= 0; --r) {
    const C dp1r = get1(r, k0 + r);
    if (r == m - 2) {
      x0 = dp0[r] + lp[r] * Ep0 + rr * E0;
      x1 = dp1r + lp[r] * Ep1 + rr * E1;
    } else {
      x0 = dp0[r] + lp[r] * Ep0 - cp[r] * x0;
      x1 = dp1r + lp[r] * Ep1 - cp[r] * x1;
    }
    if (FULL || k0 + r < Nz) {
      tile[Z.at(k0 + r, col0, lane)] = cvt<T>(x0);
      t1(k0 + r) = cvt<T>(x1);
    }
  }
}

// zsolve_pair on the pair-granular layout (ZSwzP), float, full columns (Nz = 32 MMAX, MMAX >= 4,
// lane-contiguous coefficient rows): the two right-hand sides of a row move as one 8-byte word, and
// both columns' forward values go back into the tile, so only the pivot and spike sequences stay in
// registers.  The arithmetic is zsolve_pair's, operation for operation.
template <int MMAX, typename ZS>
__device__ __forceinline__ void zsolve_pair2(float* tile, int col0, const ZS& Z, float mu, const float* sa,
                                             const float* sb, const float* sc) {
  const int lane = threadIdx.x & 31;
  constexpr int m = MMAX;
  static_assert(MMAX >= 4, "four or more rows per lane");
  constexpr int LS = MMAX + 4;
  float4 A4, B4, C4;
  auto coefs = [&](int r, float& a, float& b, float& c) {
    if ((r & 3) == 0) {
      A4 = *reinterpret_cast<const float4*>(sa + lane * LS + r);
      B4 = *reinterpret_cast<const float4*>(sb + lane * LS + r);
      C4 = *reinterpret_cast<const float4*>(sc + lane * LS + r);
    }
    a = f4_get(A4, r & 3);
    b = f4_get(B4, r & 3);
    c = f4_get(C4, r & 3);
  };
  const int k0 = lane * m;
  const unsigned full = 0xffffffffu;
  auto row = [&](int k) -> float2* { return reinterpret_cast<float2*>(tile + Z.at(k, col0, lane)); };
  float cp[MMAX], lp[MMAX];
  float rr = 0.f, cprev = 0.f, lprev = 0.f, d0prev = 0.f, d1prev = 0.f;
#pragma unroll
  for (int r = 0; r < m - 1; ++r) {
    const int k = k0 + r;
    float a, b, c;
    coefs(r, a, b, c);
    b += mu;
    const float2 d = *row(k);
    const float inv = rcp_(b - a * cprev);
    const bool last_inner = (r == m - 2);
    cp[r] = last_inner ? 0.f : c * inv;
    if (last_inner) rr = -c * inv;
    const float dp0r = (d.x - a * d0prev) * inv;
    const float dp1r = (d.y - a * d1prev) * inv;
    *row(k) = make_float2(dp0r, dp1r);
    lp[r] = ((r == 0) ? -a : -a * lprev) * inv;
    cprev = c * inv;
    d0prev = dp0r;
    d1prev = dp1r;
    lprev = lp[r];
  }
  float Dl0, Dl1, Vl, Wl, Df0, Df1, Vf, Wf;
  {
    float D0 = 0.f, D1 = 0.f, V = 0.f, W = 0.f;
#pragma unroll
    for (int r = m - 2; r >= 0; --r) {
      const float2 dr = *row(k0 + r);
      if (r == m - 2) {
        D0 = dr.x;
        D1 = dr.y;
        V = lp[r];
        W = rr;
        Dl0 = D0;
        Dl1 = D1;
        Vl = V;
        Wl = W;
      } else {
        D0 = dr.x - cp[r] * D0;
        D1 = dr.y - cp[r] * D1;
        V = lp[r] - cp[r] * V;
        W = -cp[r] * W;
      }
    }
    Df0 = D0;
    Df1 = D1;
    Vf = V;
    Wf = W;
  }
  const int kl = k0 + m - 1;
  constexpr int rl = m - 1;
  float al, bl, cl;
  if ((rl & 3) != 0) {  // the last row's group of four was loaded by the forward loop
    al = f4_get(A4, rl & 3);
    bl = f4_get(B4, rl & 3);
    cl = f4_get(C4, rl & 3);
  } else {
    coefs(rl, al, bl, cl);
  }
  bl += mu;
  const float2 dl = *row(kl);
  const float Dfn0 = __shfl_down_sync(full, Df0, 1);
  const float Dfn1 = __shfl_down_sync(full, Df1, 1);
  const float Vfn = __shfl_down_sync(full, Vf, 1);
  const float Wfn = __shfl_down_sync(full, Wf, 1);
  const bool hasn = lane < 31;
  float alpha = (lane == 0) ? 0.f : al * Vl;
  float beta = bl + al * Wl + (hasn ? cl * Vfn : 0.f);
  float gamma = hasn ? cl * Wfn : 0.f;
  float delta0 = dl.x - al * Dl0 - (hasn ? cl * Dfn0 : 0.f);
  float delta1 = dl.y - al * Dl1 - (hasn ? cl * Dfn1 : 0.f);
  // Cyclic reduction without boundary selects: at stride s, alpha is already zero on lanes < s and
  // gamma on lanes > 31 - s (lane 0 has no left and lane 31 no right coupling, and each step keeps
  // zeros within twice the stride), so k1, k2 vanish exactly where the shuffles return the lane's own
  // values, and every nonzero result equals the selected form's.
#pragma unroll
  for (int s = 1; s < 32; s <<= 1) {
    const float am = __shfl_up_sync(full, alpha, s), bm = __shfl_up_sync(full, beta, s);
    const float gm = __shfl_up_sync(full, gamma, s);
    const float dm0 = __shfl_up_sync(full, delta0, s), dm1 = __shfl_up_sync(full, delta1, s);
    const float ap = __shfl_down_sync(full, alpha, s), bp = __shfl_down_sync(full, beta, s);
    const float gp = __shfl_down_sync(full, gamma, s);
    const float dq0 = __shfl_down_sync(full, delta0, s), dq1 = __shfl_down_sync(full, delta1, s);
    const float k1 = alpha * rcp_(bm), k2 = gamma * rcp_(bp);
    const float na = -am * k1, ng = -gp * k2;
    const float nb = beta - gm * k1 - ap * k2;
    delta0 = delta0 - dm0 * k1 - dq0 * k2;
    delta1 = delta1 - dm1 * k1 - dq1 * k2;
    alpha = na;
    beta = nb;
    gamma = ng;
  }
  const float ib = rcp_(beta);
  const float E0 = delta0 * ib, E1 = delta1 * ib;
  float Ep0 = __shfl_up_sync(full, E0, 1), Ep1 = __shfl_up_sync(full, E1, 1);
  if (lane == 0) {
    Ep0 = 0.f;
    Ep1 = 0.f;
  }
  *row(kl) = make_float2(E0, E1);
  float x0 = E0, x1 = E1;
#pragma unroll
  for (int r = m - 2; r >= 0; --r) {
    const float2 dr = *row(k0 + r);
    if (r == m - 2) {
      x0 = dr.x + lp[r] * Ep0 + rr * E0;
      x1 = dr.y + lp[r] * Ep1 + rr * E1;
    } else {
      x0 = dr.x + lp[r] * Ep0 - cp[r] * x0;
      x1 = dr.y + lp[r] * Ep1 - cp[r] * x1;
    }
    *row(k0 + r) = make_float2(x0, x1);
  }
}

}  // namespace cans
