// Shared-memory line transforms for the x and y passes of the eigenfunction-expansion solver
// (the operator F^{x_i} of Eq. poi_reduced: real DFT for periodic, DCT-II/DST-II for Neumann /
// Dirichlet walls, with the inverses DFT^-1, DCT-III, DST-III; DCT-IV / DST-IV, their own inverses,
// for a Neumann wall paired with a Dirichlet wall).
//
// A CTA holds `nl` lines (nl a power of two) of N = 2M reals in shared memory.  Each real line is
// packed into M complex numbers (even -> real part, odd -> imaginary part), transformed by a
// mixed-radix (2, 3, 4, 8) Stockham FFT of length M, and post-processed into the N real
// coefficients (the standard half-length real-FFT split, plus Makhoul's 1980 reordering and
// quarter-wave twiddle for the cosine/sine transforms).  Complex element m of line l lives at
// m*(nl+1) + l: lines are interleaved so that lanes of a warp that work on different lines at the
// same m hit consecutive banks, and the one-cell row padding spreads the copy phases (consecutive
// samples of one line) over all banks.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cans {

enum { BC_P = 0, BC_NN = 1, BC_DD = 2, BC_ND = 3, BC_DN = 4 };  // ND / DN: z only (mixed walls)
// wall rule at the low and the high end of a walled direction
__host__ __device__ __forceinline__ int bc_lo(int bc) { return bc == BC_ND ? BC_NN : (bc == BC_DN ? BC_DD : bc); }
__host__ __device__ __forceinline__ int bc_hi(int bc) { return bc == BC_ND ? BC_DD : (bc == BC_DN ? BC_NN : bc); }

template <typename T> struct V2;
template <> struct V2<float> { typedef float2 t; };
template <> struct V2<double> { typedef double2 t; };

template <typename T> __device__ __forceinline__ typename V2<T>::t mk2(T x, T y) {
  typename V2<T>::t r;
  r.x = x;
  r.y = y;
  return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = fma(a.x, b.x, -a.y * b.y);
  r.y = fma(a.x, b.y, a.y * b.x);
  return r;
}
template <typename C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
// multiply by -i
template <typename C> __device__ __forceinline__ C cmi(C a) { C r; r.x = a.y; r.y = -a.x; return r; }

// Per-direction line-transform tables (device pointers) and the FFT factorisation of M = N/2.
template <typename T>
struct LineTab {
  const typename V2<T>::t* tw;    // M entries: exp(-2 pi i t / M)
  const typename V2<T>::t* post;  // M+1 entries: exp(-2 pi i k / N)
  const typename V2<T>::t* mak;   // M+1 entries: exp(-i pi k / (2N))
  // per-stage twiddles of the warp-per-line engine (wline.cuh), stage by stage in [r][k] order so
  // that the lanes of a warp read consecutive entries; null when the engine does not take M
  const typename V2<T>::t* wst = nullptr;
  int n, m, bc, nst;
  int radix[16];
};

struct Lay {
  int nl;  // lines in the tile (power of two); rows are padded to nl + 1 complex cells
  __device__ __forceinline__ int c(int m, int l) const { return m * (nl + 1) + l; }
  // real slot s of line l inside the same storage (two reals per complex cell)
  __device__ __forceinline__ int r(int s, int l) const { return 2 * c(s >> 1, l) + (s & 1); }
};

// Quarter-wave lines (a Neumann wall paired with a Dirichlet wall).  The cosine transform
//   Y_k = 2 sum_n x_n cos(pi (2n+1)(2k+1) / 4N)  (DCT-IV)
// runs as one half-length complex FFT between two twiddles:
//   z_m = (x_2m + i x_{N-1-2m}) exp(-i pi (4m+1)/4N),  Z = FFT_M(z),  u_k = Z_k exp(-i pi k/N),
//   Y_2k = 2 Re u_k,  Y_{N-1-2k} = -2 Im u_k.
// The sine transform (DST-IV, Dirichlet wall first) is the cosine one of (-1)^n x_n read backwards.
// Both are their own inverses up to 2N, so the inverse pass (times N) is the same routine with
// factor 1.  The direction's tables then hold mak[m] = exp(-i pi (4m+1)/4N) (pre) and
// post[k] = exp(-i pi k/N) (post).
__host__ __device__ __forceinline__ bool quarter(int bc) { return bc == BC_ND || bc == BC_DN; }
// sign of sample (or slot) n on the way into the half-length FFT: Dirichlet-first lines alternate
__host__ __device__ __forceinline__ bool neg_in(int bc, int n) { return (bc == BC_DD || bc == BC_DN) && (n & 1); }

// position of input sample n inside the sequence fed to the half-length FFT
//   periodic: identity.  Neumann / Dirichlet (Makhoul): even samples first in order, odd samples
//   after them in reverse order.  Quarter-wave: x_2m is the real part of z_m, x_{N-1-2m} its
//   imaginary part (odd n sits at position N - n).
__device__ __forceinline__ int perm_in(int bc, int N, int n) {
  if (bc == BC_P) return n;
  if (quarter(bc)) return (n & 1) ? N - n : n;
  return (n & 1) ? (N - 1 - (n >> 1)) : (n >> 1);
}

// the two samples (or slots) that pack into complex element m of a quarter-wave line, and the two
// that complex output k of the half-length FFT produces (in the same order: real, imaginary part)
__device__ __forceinline__ void qw_pair(int bc, int N, int m, int& a, int& b) {
  a = 2 * m;
  b = N - 1 - 2 * m;
  if (bc == BC_DN) {  // read backwards
    const int t = a;
    a = b;
    b = t;
  }
}

// ---- small DFTs (forward sign) --------------------------------------------------------------
template <int R, typename C> struct Dft;
template <typename C> struct Dft<2, C> {
  static __device__ __forceinline__ void run(C* v) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};
template <typename C> struct Dft<3, C> {
  static __device__ __forceinline__ void run(C* v) {
    typedef decltype(v[0].x) T;
    const T c1 = (T)-0.5, s1 = (T)-0.86602540378443864676372317075294;  // exp(-2 pi i/3)
    C t = cadd(v[1], v[2]), u = csub(v[1], v[2]);
    C y0 = cadd(v[0], t);
    C m;
    m.x = fma(c1, t.x, v[0].x);
    m.y = fma(c1, t.y, v[0].y);
    C su;  // i * s1 * u
    su.x = -s1 * u.y;
    su.y = s1 * u.x;
    v[0] = y0;
    v[1] = cadd(m, su);
    v[2] = csub(m, su);
  }
};
template <typename C> struct Dft<4, C> {
  static __device__ __forceinline__ void run(C* v) {
    C a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    C c = cadd(v[1], v[3]), d = cmi(csub(v[1], v[3]));
    v[0] = cadd(a, c);
    v[2] = csub(a, c);
    v[1] = cadd(b, d);
    v[3] = csub(b, d);
  }
};
template <typename C> struct Dft<8, C> {
  static __device__ __forceinline__ void run(C* v) {
    typedef decltype(v[0].x) T;
    const T r = (T)0.70710678118654752440084436210485;
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    Dft<4, C>::run(e);
    Dft<4, C>::run(o);
    // twiddles exp(-i pi k/4), k = 1, 2, 3
    C o1;
    o1.x = r * (o[1].x + o[1].y);
    o1.y = r * (o[1].y - o[1].x);
    C o2 = cmi(o[2]);
    C o3;
    o3.x = r * (o[3].y - o[3].x);
    o3.y = -r * (o[3].x + o[3].y);
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
  }
};

// One Stockham radix-R stage over all nl lines, in place in shared memory.  Every thread first
// loads and transforms its butterflies into registers, the CTA synchronises, then every thread
// stores.  Requires nl*M <= MAXV*blockDim.x.
template <int R, int MAXV, typename T>
__device__ __forceinline__ void fft_stage(typename V2<T>::t* buf, const Lay& L, int lognl, int M, int Ns,
                                          const typename V2<T>::t* __restrict__ tw) {
  typedef typename V2<T>::t C;
  constexpr int Q = (MAXV + R - 1) / R;
  const int nb = M / R;
  const int total = nb << lognl;
  const int tstride = M / (Ns * R);
  C v[Q][R];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int t = threadIdx.x + q * blockDim.x;
    if (t < total) {
      const int l = t & (L.nl - 1), j = t >> lognl;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = buf[L.c(j + r * nb, l)];
      if (Ns > 1) {
        const int k = j % Ns;
        const int st = tstride * k;
#pragma unroll
        for (int r = 1; r < R; ++r) v[q][r] = cmul(v[q][r], __ldg(&tw[r * st]));
      }
      Dft<R, C>::run(v[q]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int t = threadIdx.x + q * blockDim.x;
    if (t < total) {
      const int l = t & (L.nl - 1), j = t >> lognl;
      const int k = j % Ns;
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[L.c(base + r * Ns, l)] = v[q][r];
    }
  }
  __syncthreads();
}

// ---- compile-time radix schedule for M = 2^a 3^b: threes first, then eights, then a 4 or a 2 ----
__host__ __device__ constexpr int m_threes(int M) {
  int n = 0;
  while (M > 1 && M % 3 == 0) { M /= 3; ++n; }
  return n;
}
__host__ __device__ constexpr int m_twos(int M) {
  while (M > 1 && M % 3 == 0) M /= 3;
  int n = 0;
  while (M > 1 && M % 2 == 0) { M /= 2; ++n; }
  return n;
}
__host__ __device__ constexpr int m_nst(int M) { return m_threes(M) + m_twos(M) / 3 + ((m_twos(M) % 3) ? 1 : 0); }
__host__ __device__ constexpr int m_radix(int M, int s) {
  return (s < m_threes(M)) ? 3 : (s < m_threes(M) + m_twos(M) / 3) ? 8 : ((m_twos(M) % 3 == 2) ? 4 : 2);
}
__host__ __device__ constexpr int m_ns(int M, int s) {
  int p = 1;
  for (int i = 0; i < s; ++i) p *= m_radix(M, i);
  return p;
}

// Stage with compile-time length and stride (all index arithmetic folds to shifts and multiplies).
template <int R, int MAXV, typename T, int M, int Ns>
__device__ __forceinline__ void fft_stage_ct(typename V2<T>::t* buf, const Lay& L, int lognl,
                                             const typename V2<T>::t* __restrict__ tw) {
  typedef typename V2<T>::t C;
  constexpr int Q = (MAXV + R - 1) / R;
  constexpr int nb = M / R;
  constexpr int tstride = M / (Ns * R);
  const int total = nb << lognl;
  C v[Q][R];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int t = threadIdx.x + q * blockDim.x;
    if (t < total) {
      const int l = t & (L.nl - 1), j = t >> lognl;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = buf[L.c(j + r * nb, l)];
      if (Ns > 1) {
        const int k = j % Ns;
        const int st = tstride * k;
#pragma unroll
        for (int r = 1; r < R; ++r) v[q][r] = cmul(v[q][r], __ldg(&tw[r * st]));
      }
      Dft<R, C>::run(v[q]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int t = threadIdx.x + q * blockDim.x;
    if (t < total) {
      const int l = t & (L.nl - 1), j = t >> lognl;
      const int k = j % Ns;
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[L.c(base + r * Ns, l)] = v[q][r];
    }
  }
  __syncthreads();
}

template <int MAXV, typename T, int M, int S, int NST>
struct FftStages {
  static __device__ __forceinline__ void run(typename V2<T>::t* buf, const Lay& L, int lognl,
                                             const typename V2<T>::t* tw) {
    fft_stage_ct<m_radix(M, S), MAXV, T, M, m_ns(M, S)>(buf, L, lognl, tw);
    FftStages<MAXV, T, M, S + 1, NST>::run(buf, L, lognl, tw);
  }
};
template <int MAXV, typename T, int M, int NST>
struct FftStages<MAXV, T, M, NST, NST> {
  static __device__ __forceinline__ void run(typename V2<T>::t*, const Lay&, int, const typename V2<T>::t*) {}
};

template <int MAXV, typename T, int MC = 0>
__device__ __forceinline__ void fft_lines(typename V2<T>::t* buf, const Lay& L, int lognl, const LineTab<T>& tb) {
  if (MC > 0) {
    FftStages<MAXV, T, MC, 0, m_nst(MC)>::run(buf, L, lognl, tb.tw);
    return;
  }
  int Ns = 1;
  for (int s = 0; s < tb.nst; ++s) {
    const int R = tb.radix[s];
    if (R == 8)
      fft_stage<8, MAXV, T>(buf, L, lognl, tb.m, Ns, tb.tw);
    else if (R == 4)
      fft_stage<4, MAXV, T>(buf, L, lognl, tb.m, Ns, tb.tw);
    else if (R == 3)
      fft_stage<3, MAXV, T>(buf, L, lognl, tb.m, Ns, tb.tw);
    else
      fft_stage<2, MAXV, T>(buf, L, lognl, tb.m, Ns, tb.tw);
    Ns *= R;
  }
}

// Output slots of the pair (k, M-k) of the forward post-processing (-1 = none).
__device__ __forceinline__ void fwd_slots(int bc, int N, int M, int k, int s[4]) {
  s[0] = s[1] = s[2] = s[3] = -1;
  if (bc == BC_P) {
    if (k == 0) { s[0] = 0; s[1] = 1; }
    else {
      s[0] = 2 * k; s[1] = 2 * k + 1;
      if (k != M - k) { s[2] = 2 * (M - k); s[3] = 2 * (M - k) + 1; }
    }
  } else {
    if (k == 0) { s[0] = 0; s[1] = M; }
    else {
      s[0] = k; s[1] = N - k;
      if (k != M - k) { s[2] = M - k; s[3] = M + k; }
    }
    if (bc == BC_DD) {
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (s[e] >= 0) s[e] = N - 1 - s[e];
    }
  }
}

// Forward post-processing: buf holds FFT_M of the packed line; afterwards the storage holds the N
// real output slots (read with Lay::r).  Pairs (k, M-k) are handled together:
//   V_k = E_k + exp(-2 pi i k/N) O_k with E, O the even/odd half spectra (real-FFT split);
//   periodic: slots carry Re/Im V_k;  cosine: Y_k = 2 Re(W^k V_k), Y_{N-k} = -2 Im(W^k V_k),
//   W = exp(-i pi/(2N)) (Makhoul);  sine: the cosine result of the sign-alternated input, reversed.
template <int MAXV, typename T, int MC = 0>
__device__ __forceinline__ void post_forward(typename V2<T>::t* buf, const Lay& L, int lognl, const LineTab<T>& tb) {
  typedef typename V2<T>::t C;
  constexpr int J = MAXV / 2 + 2;
  const int M = MC > 0 ? MC : tb.m, N = 2 * M, half = M >> 1;
  const int total = (half + 1) << lognl;
  T val[J][4];
  T* bufT = reinterpret_cast<T*>(buf);
#pragma unroll
  for (int q = 0; q < J; ++q) {
    const int t = threadIdx.x + q * blockDim.x;
    if (t < total) {
      const int l = t & (L.nl - 1), k = t >> lognl;
      if (k == 0) {
        const C z = buf[L.c(0, l)];
        const T v0 = z.x + z.y, vm = z.x - z.y;
        if (tb.bc == BC_P) {
          val[q][0] = v0;
          val[q][1] = vm;
        } else {
          val[q][0] = (T)2 * v0;
          val[q][1] = (T)1.41421356237309504880168872420970 * vm;
        }
        val[q][2] = val[q][3] = (T)0;
      } else {
        const C zk = buf[L.c(k, l)], zm = buf[L.c(M - k, l)];
        C E, O;
        E.x = (T)0.5 * (zk.x + zm.x);
        E.y = (T)0.5 * (zk.y - zm.y);
        O.x = (T)0.5 * (zk.y + zm.y);
        O.y = (T)-0.5 * (zk.x - zm.x);
        const C wO = cmul(__ldg(&tb.post[k]), O);
        const C vk = cadd(E, wO);
        const C vmk = cconj(csub(E, wO));
        if (tb.bc == BC_P) {
          val[q][0] = vk.x;
          val[q][1] = vk.y;
          val[q][2] = vmk.x;
          val[q][3] = vmk.y;
        } else {
          const C a = cmul(__ldg(&tb.mak[k]), vk);
          const C b = cmul(__ldg(&tb.mak[M - k]), vmk);
          val[q][0] = (T)2 * a.x;
          val[q][1] = (T)-2 * a.y;
          val[q][2] = (T)2 * b.x;
          val[q][3] = (T)-2 * b.y;
        }
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < J; ++q) {
    const int t = threadIdx.x + q * blockDim.x;
    if (t < total) {
      const int l = t & (L.nl - 1), k = t >> lognl;
      int s[4];
      fwd_slots(tb.bc, N, M, k, s);
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (s[e] >= 0) bufT[L.r(s[e], l)] = val[q][e];
    }
  }
  __syncthreads();
}

// Inverse pre-processing: storage holds the N real slots; afterwards buf holds conj(Z) where
// IFFT_M(Z) is the packed line times N (the caller runs the forward FFT and conjugates back).
//   periodic: Z_k = (X_k + conj X_{M-k}) + i exp(2 pi i k/N) (X_k - conj X_{M-k});
//   cosine / sine: first V_k = W^{-k} (Y_k - i Y_{N-k}) / 2, then the same with X = V.
template <int MAXV, typename T, int MC = 0>
__device__ __forceinline__ void pre_inverse(typename V2<T>::t* buf, const Lay& L, int lognl, const LineTab<T>& tb) {
  typedef typename V2<T>::t C;
  constexpr int J = MAXV / 2 + 2;
  const int M = MC > 0 ? MC : tb.m, N = 2 * M, half = M >> 1;
  const int total = (half + 1) << lognl;
  C zk_out[J], zm_out[J];
  const T* bufT = reinterpret_cast<const T*>(buf);
  const bool dd = (tb.bc == BC_DD);
#pragma unroll
  for (int q = 0; q < J; ++q) {
    const int t = threadIdx.x + q * blockDim.x;
    if (t < total) {
      const int l = t & (L.nl - 1), k = t >> lognl;
      C xk, xm;
      if (tb.bc == BC_P) {
        if (k == 0) {
          xk = mk2<T>(bufT[L.r(0, l)], (T)0);
          xm = mk2<T>(bufT[L.r(1, l)], (T)0);  // X_M
        } else {
          xk = mk2<T>(bufT[L.r(2 * k, l)], bufT[L.r(2 * k + 1, l)]);
          xm = mk2<T>(bufT[L.r(2 * (M - k), l)], bufT[L.r(2 * (M - k) + 1, l)]);
        }
      } else {
#define SLOT(q_) (dd ? (N - 1 - (q_)) : (q_))
        if (k == 0) {
          xk = mk2<T>((T)0.5 * bufT[L.r(SLOT(0), l)], (T)0);
          xm = mk2<T>((T)0.70710678118654752440084436210485 * bufT[L.r(SLOT(M), l)], (T)0);  // V_M
        } else {
          const C yk = mk2<T>((T)0.5 * bufT[L.r(SLOT(k), l)], (T)-0.5 * bufT[L.r(SLOT(N - k), l)]);
          const C ym = mk2<T>((T)0.5 * bufT[L.r(SLOT(M - k), l)], (T)-0.5 * bufT[L.r(SLOT(M + k), l)]);
          xk = cmul(cconj(__ldg(&tb.mak[k])), yk);
          xm = cmul(cconj(__ldg(&tb.mak[M - k])), ym);
        }
#undef SLOT
      }
      if (k == 0) {
        zk_out[q] = mk2<T>(xk.x + xm.x, xk.x - xm.x);
      } else {
        const C A = cadd(xk, cconj(xm));
        const C B = csub(xk, cconj(xm));
        const C wB = cmul(cconj(__ldg(&tb.post[k])), B);  // exp(+2 pi i k/N) B
        const C iwB = mk2<T>(-wB.y, wB.x);                 // times i
        zk_out[q] = cadd(A, iwB);
        zm_out[q] = cconj(csub(A, iwB));
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < J; ++q) {
    const int t = threadIdx.x + q * blockDim.x;
    if (t < total) {
      const int l = t & (L.nl - 1), k = t >> lognl;
      buf[L.c(k, l)] = cconj(zk_out[q]);
      if (k != 0 && k != M - k) buf[L.c(M - k, l)] = cconj(zm_out[q]);
    }
  }
  __syncthreads();
}

// Value of output sample n of the inverse transform (times N), after pre_inverse + fft_lines.
template <typename T, int MC = 0>
__device__ __forceinline__ T inverse_sample(const typename V2<T>::t* buf, const Lay& L, const LineTab<T>& tb, int n,
                                            int l) {
  const int N = MC > 0 ? 2 * MC : tb.n;
  if (quarter(tb.bc) && N >= 2) {  // post-twiddle of the complex output that carries sample n
    const int nn = (tb.bc == BC_DN) ? N - 1 - n : n;  // its index in the cosine form
    const int k = (nn & 1) ? (N - 1 - nn) >> 1 : nn >> 1;
    const typename V2<T>::t u = cmul(buf[L.c(k, l)], __ldg(&tb.post[k]));
    return (nn & 1) ? -u.y : u.x;
  }
  const int s = perm_in(tb.bc, N, n);
  const T* bufT = reinterpret_cast<const T*>(buf);
  T v = bufT[L.r(s, l)];
  if (s & 1) v = -v;  // conjugate back
  if (tb.bc == BC_DD && (n & 1)) v = -v;
  return v;
}

// Store input sample n of line l (forward transform) into the packed position.
template <typename T, int MC = 0>
__device__ __forceinline__ void forward_store(typename V2<T>::t* buf, const Lay& L, const LineTab<T>& tb, int n, int l,
                                              T v) {
  const int s = perm_in(tb.bc, MC > 0 ? 2 * MC : tb.n, n);
  if (neg_in(tb.bc, n)) v = -v;
  reinterpret_cast<T*>(buf)[L.r(s, l)] = v;
}

// ---- fused variants: first stage reads the staged input directly, last step writes to global -------
// sample index n of a line whose value sits at position s of the half-length FFT's real input
__device__ __forceinline__ int perm_out(int bc, int N, int s) {
  if (bc == BC_P) return s;
  return (s < (N >> 1)) ? 2 * s : 2 * (N - 1 - s) + 1;
}

// Stockham stage 1 (stride 1) with its inputs fetched through load(l, n) (real sample n of line l):
// the packed complex z_m = (v_2m, v_2m+1) of the permuted sequence v is assembled on the fly.
template <int R, int MAXV, typename T, int M, typename LoadF>
__device__ __forceinline__ void fft_stage1_loaded(typename V2<T>::t* buf, const Lay& L, int lognl, int bc,
                                                  LoadF load, const typename V2<T>::t* __restrict__ qpre) {
  typedef typename V2<T>::t C;
  constexpr int Q = (MAXV + R - 1) / R;
  constexpr int nb = M / R;
  constexpr int N = 2 * M;
  const int total = nb << lognl;
  C v[Q][R];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int t = threadIdx.x + q * blockDim.x;
    if (t < total) {
      const int l = t & (L.nl - 1), j = t >> lognl;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int m = j + r * nb;
        int n0, n1;
        if (quarter(bc)) {
          n0 = 2 * m;
          n1 = N - 1 - 2 * m;
        } else {
          n0 = perm_out(bc, N, 2 * m);
          n1 = perm_out(bc, N, 2 * m + 1);
        }
        T x0 = load(l, n0), x1 = load(l, n1);
        if (neg_in(bc, n0)) x0 = -x0;
        if (neg_in(bc, n1)) x1 = -x1;
        v[q][r] = mk2<T>(x0, x1);
        if (quarter(bc)) v[q][r] = cmul(v[q][r], __ldg(&qpre[m]));
      }
      Dft<R, C>::run(v[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int t = threadIdx.x + q * blockDim.x;
    if (t < total) {
      const int l = t & (L.nl - 1), j = t >> lognl;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[L.c(j * R + r, l)] = v[q][r];
    }
  }
  __syncthreads();
}

// Forward post-processing whose N output slots go straight to store(l, slot, value).
// JFAST: consecutive threads take consecutive k of one line (coalesced stores along contiguous
// lines); otherwise consecutive threads take consecutive lines at one k (strided lines).
template <int MAXV, typename T, int M, bool JFAST = false, typename StoreF>
__device__ __forceinline__ void post_forward_store(const typename V2<T>::t* buf, const Lay& L, int lognl,
                                                   const LineTab<T>& tb, StoreF store) {
  typedef typename V2<T>::t C;
  constexpr int N = 2 * M, half = M >> 1;
  if (quarter(tb.bc)) {
    for (int t = threadIdx.x; t < (M << lognl); t += blockDim.x) {
      const int l = JFAST ? t / M : (t & (L.nl - 1));
      const int k = JFAST ? t - l * M : (t >> lognl);
      const C u = cmul(buf[L.c(k, l)], __ldg(&tb.post[k]));
      int a, b;
      qw_pair(tb.bc, N, k, a, b);
      store(l, a, (T)2 * u.x);
      store(l, b, (T)-2 * u.y);
    }
    return;
  }
  const int total = (half + 1) << lognl;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int l = JFAST ? t / (half + 1) : (t & (L.nl - 1));
    const int k = JFAST ? t - l * (half + 1) : (t >> lognl);
    T val[4];
    if (k == 0) {
      const C z = buf[L.c(0, l)];
      const T v0 = z.x + z.y, vm = z.x - z.y;
      if (tb.bc == BC_P) {
        val[0] = v0;
        val[1] = vm;
      } else {
        val[0] = (T)2 * v0;
        val[1] = (T)1.41421356237309504880168872420970 * vm;
      }
      val[2] = val[3] = (T)0;
    } else {
      const C zk = buf[L.c(k, l)], zm = buf[L.c(M - k, l)];
      C E, O;
      E.x = (T)0.5 * (zk.x + zm.x);
      E.y = (T)0.5 * (zk.y - zm.y);
      O.x = (T)0.5 * (zk.y + zm.y);
      O.y = (T)-0.5 * (zk.x - zm.x);
      const C wO = cmul(__ldg(&tb.post[k]), O);
      const C vk = cadd(E, wO);
      const C vmk = cconj(csub(E, wO));
      if (tb.bc == BC_P) {
        val[0] = vk.x;
        val[1] = vk.y;
        val[2] = vmk.x;
        val[3] = vmk.y;
      } else {
        const C a = cmul(__ldg(&tb.mak[k]), vk);
        const C b = cmul(__ldg(&tb.mak[M - k]), vmk);
        val[0] = (T)2 * a.x;
        val[1] = (T)-2 * a.y;
        val[2] = (T)2 * b.x;
        val[3] = (T)-2 * b.y;
      }
    }
    int sl[4];
    fwd_slots(tb.bc, N, M, k, sl);
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (sl[e] >= 0) store(l, sl[e], val[e]);
  }
}

// Inverse pre-processing whose input slots come from loadslot(l, slot) (no read of buf), writing
// conj(Z) into buf; the caller then runs the FFT stages.
template <int MAXV, typename T, int M, typename LoadF>
__device__ __forceinline__ void pre_inverse_loaded(typename V2<T>::t* buf, const Lay& L, int lognl,
                                                   const LineTab<T>& tb, LoadF loadslot) {
  typedef typename V2<T>::t C;
  constexpr int N = 2 * M, half = M >> 1;
  if (quarter(tb.bc)) {
    for (int t = threadIdx.x; t < (M << lognl); t += blockDim.x) {
      const int l = t & (L.nl - 1), m = t >> lognl;
      const int a = 2 * m, b = N - 1 - 2 * m;
      T xa = loadslot(l, a), xb = loadslot(l, b);
      if (neg_in(tb.bc, a)) xa = -xa;
      if (neg_in(tb.bc, b)) xb = -xb;
      buf[L.c(m, l)] = cmul(mk2<T>(xa, xb), __ldg(&tb.mak[m]));
    }
    __syncthreads();
    return;
  }
  const int total = (half + 1) << lognl;
  const bool dd = (tb.bc == BC_DD);
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int l = t & (L.nl - 1), k = t >> lognl;
    C xk, xm;
    if (tb.bc == BC_P) {
      if (k == 0) {
        xk = mk2<T>(loadslot(l, 0), (T)0);
        xm = mk2<T>(loadslot(l, 1), (T)0);
      } else {
        xk = mk2<T>(loadslot(l, 2 * k), loadslot(l, 2 * k + 1));
        xm = mk2<T>(loadslot(l, 2 * (M - k)), loadslot(l, 2 * (M - k) + 1));
      }
    } else {
#define SLOT(q_) (dd ? (N - 1 - (q_)) : (q_))
      if (k == 0) {
        xk = mk2<T>((T)0.5 * loadslot(l, SLOT(0)), (T)0);
        xm = mk2<T>((T)0.70710678118654752440084436210485 * loadslot(l, SLOT(M)), (T)0);
      } else {
        const C yk = mk2<T>((T)0.5 * loadslot(l, SLOT(k)), (T)-0.5 * loadslot(l, SLOT(N - k)));
        const C ym = mk2<T>((T)0.5 * loadslot(l, SLOT(M - k)), (T)-0.5 * loadslot(l, SLOT(M + k)));
        xk = cmul(cconj(__ldg(&tb.mak[k])), yk);
        xm = cmul(cconj(__ldg(&tb.mak[M - k])), ym);
      }
#undef SLOT
    }
    if (k == 0) {
      buf[L.c(0, l)] = cconj(mk2<T>(xk.x + xm.x, xk.x - xm.x));
    } else {
      const C A = cadd(xk, cconj(xm));
      const C B = csub(xk, cconj(xm));
      const C wB = cmul(cconj(__ldg(&tb.post[k])), B);
      const C iwB = mk2<T>(-wB.y, wB.x);
      buf[L.c(k, l)] = cconj(cadd(A, iwB));
      if (k != M - k) buf[L.c(M - k, l)] = csub(A, iwB);  // conj(conj(A - i w B))
    }
  }
  __syncthreads();
}

// Last Stockham stage of the inverse transform with its outputs sent to store(l, n, value): the
// conjugate-back and the unpacking of z_m into samples 2m, 2m+1 of v (and v -> x) are fused.
template <int R, int MAXV, typename T, int M, int Ns, bool JFAST = false, typename StoreF>
__device__ __forceinline__ void fft_last_stage_store(const typename V2<T>::t* buf, const Lay& L, int lognl, int bc,
                                                     const typename V2<T>::t* __restrict__ tw, StoreF store,
                                                     const typename V2<T>::t* __restrict__ qpost) {
  typedef typename V2<T>::t C;
  constexpr int Q = (MAXV + R - 1) / R;
  constexpr int nb = M / R;
  constexpr int tstride = M / (Ns * R);
  constexpr int N = 2 * M;
  const int total = nb << lognl;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int t = threadIdx.x + q * blockDim.x;
    if (t < total) {
      const int l = JFAST ? t / nb : (t & (L.nl - 1));
      const int j = JFAST ? t - l * nb : (t >> lognl);
      C v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = buf[L.c(j + r * nb, l)];
      const int k = j % Ns;
      if (Ns > 1) {
        const int st = tstride * k;
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmul(v[r], __ldg(&tw[r * st]));
      }
      Dft<R, C>::run(v);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int m = base + r * Ns;
        if (quarter(bc)) {  // post-twiddle; the FFT ran forward on the pre-twiddled slots
          const C u = cmul(v[r], __ldg(&qpost[m]));
          int a, b;
          qw_pair(bc, N, m, a, b);
          store(l, a, u.x);
          store(l, b, -u.y);
          continue;
        }
        const int n0 = perm_out(bc, N, 2 * m), n1 = perm_out(bc, N, 2 * m + 1);
        T x0 = v[r].x, x1 = -v[r].y;  // conjugate back
        if (bc == BC_DD) {
          if (n0 & 1) x0 = -x0;
          if (n1 & 1) x1 = -x1;
        }
        store(l, n0, x0);
        store(l, n1, x1);
      }
    }
  }
}

template <int MAXV, typename T, int M, int S, int NST>
struct FftStagesButLast {
  static __device__ __forceinline__ void run(typename V2<T>::t* buf, const Lay& L, int lognl,
                                             const typename V2<T>::t* tw) {
    if (S < NST - 1) {
      fft_stage_ct<m_radix(M, S), MAXV, T, M, m_ns(M, S)>(buf, L, lognl, tw);
      FftStagesButLast<MAXV, T, M, (S + 1 < NST ? S + 1 : NST), NST>::run(buf, L, lognl, tw);
    }
  }
};
template <int MAXV, typename T, int M, int NST>
struct FftStagesButLast<MAXV, T, M, NST, NST> {
  static __device__ __forceinline__ void run(typename V2<T>::t*, const Lay&, int, const typename V2<T>::t*) {}
};

// Whole forward line transform from a loader to a slot store (M compile time, M >= 2).
template <int MAXV, typename T, int M, bool JFAST = false, typename LoadF, typename StoreF>
__device__ __forceinline__ void line_forward_fused(typename V2<T>::t* buf, const Lay& L, int lognl,
                                                   const LineTab<T>& tb, LoadF load, StoreF store) {
  constexpr int NST = m_nst(M);
  fft_stage1_loaded<m_radix(M, 0), MAXV, T, M>(buf, L, lognl, tb.bc, load, tb.mak);
  FftStages<MAXV, T, M, 1, NST>::run(buf, L, lognl, tb.tw);
  post_forward_store<MAXV, T, M, JFAST>(buf, L, lognl, tb, store);
}

// Whole inverse line transform from a slot loader to a sample store (M compile time, M >= 2).
template <int MAXV, typename T, int M, bool JFAST = false, typename LoadF, typename StoreF>
__device__ __forceinline__ void line_inverse_fused(typename V2<T>::t* buf, const Lay& L, int lognl,
                                                   const LineTab<T>& tb, LoadF loadslot, StoreF store) {
  constexpr int NST = m_nst(M);
  pre_inverse_loaded<MAXV, T, M>(buf, L, lognl, tb, loadslot);
  FftStagesButLast<MAXV, T, M, 0, NST>::run(buf, L, lognl, tb.tw);
  fft_last_stage_store<m_radix(M, NST - 1), MAXV, T, M, m_ns(M, NST - 1), JFAST>(buf, L, lognl, tb.bc, tb.tw,
                                                                                 store, tb.post);
}

// ---- quarter-wave steps on a staged tile ----------------------------------------------------------
// pre-twiddle of the packed elements (each thread scales its own cells)
template <typename T, int MC = 0>
__device__ __forceinline__ void qw_pretwiddle(typename V2<T>::t* buf, const Lay& L, int lognl, const LineTab<T>& tb) {
  const int M = MC > 0 ? MC : tb.m;
  for (int t = threadIdx.x; t < (M << lognl); t += blockDim.x) {
    const int l = t & (L.nl - 1), m = t >> lognl;
    buf[L.c(m, l)] = cmul(buf[L.c(m, l)], __ldg(&tb.mak[m]));
  }
  __syncthreads();
}

// forward post-twiddle: the N slots of the line, every k written after every thread has read
template <int MAXV, typename T, int MC = 0>
__device__ __forceinline__ void qw_post_forward(typename V2<T>::t* buf, const Lay& L, int lognl, const LineTab<T>& tb) {
  typedef typename V2<T>::t C;
  constexpr int J = MAXV + 1;
  const int M = MC > 0 ? MC : tb.m, N = 2 * M;
  const int total = M << lognl;
  C u[J];
#pragma unroll
  for (int q = 0; q < J; ++q) {
    const int t = threadIdx.x + q * blockDim.x;
    if (t < total) {
      const int l = t & (L.nl - 1), k = t >> lognl;
      u[q] = cmul(buf[L.c(k, l)], __ldg(&tb.post[k]));
    }
  }
  __syncthreads();
  T* bufT = reinterpret_cast<T*>(buf);
#pragma unroll
  for (int q = 0; q < J; ++q) {
    const int t = threadIdx.x + q * blockDim.x;
    if (t < total) {
      const int l = t & (L.nl - 1), k = t >> lognl;
      int a, b;
      qw_pair(tb.bc, N, k, a, b);
      bufT[L.r(a, l)] = (T)2 * u[q].x;
      bufT[L.r(b, l)] = (T)-2 * u[q].y;
    }
  }
  __syncthreads();
}

// inverse pre-step: the slots of the line (in the real storage) packed and pre-twiddled into buf
template <int MAXV, typename T, int MC = 0>
__device__ __forceinline__ void qw_pre_inverse(typename V2<T>::t* buf, const Lay& L, int lognl, const LineTab<T>& tb) {
  typedef typename V2<T>::t C;
  constexpr int J = MAXV + 1;
  const int M = MC > 0 ? MC : tb.m, N = 2 * M;
  const int total = M << lognl;
  const T* bufT = reinterpret_cast<const T*>(buf);
  C z[J];
#pragma unroll
  for (int q = 0; q < J; ++q) {
    const int t = threadIdx.x + q * blockDim.x;
    if (t < total) {
      const int l = t & (L.nl - 1), m = t >> lognl;
      const int a = 2 * m, b = N - 1 - 2 * m;
      T xa = bufT[L.r(a, l)], xb = bufT[L.r(b, l)];
      if (neg_in(tb.bc, a)) xa = -xa;
      if (neg_in(tb.bc, b)) xb = -xb;
      z[q] = cmul(mk2<T>(xa, xb), __ldg(&tb.mak[m]));
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < J; ++q) {
    const int t = threadIdx.x + q * blockDim.x;
    if (t < total) {
      const int l = t & (L.nl - 1), m = t >> lognl;
      buf[L.c(m, l)] = z[q];
    }
  }
  __syncthreads();
}

template <int MAXV, typename T, int MC = 0>
__device__ __forceinline__ void line_forward(typename V2<T>::t* buf, const Lay& L, int lognl, const LineTab<T>& tb) {
  if (MC == 0 && tb.n < 2) return;
  if (quarter(tb.bc)) {
    qw_pretwiddle<T, MC>(buf, L, lognl, tb);
    fft_lines<MAXV, T, MC>(buf, L, lognl, tb);
    qw_post_forward<MAXV, T, MC>(buf, L, lognl, tb);
    return;
  }
  fft_lines<MAXV, T, MC>(buf, L, lognl, tb);
  post_forward<MAXV, T, MC>(buf, L, lognl, tb);
}

template <int MAXV, typename T, int MC = 0>
__device__ __forceinline__ void line_inverse(typename V2<T>::t* buf, const Lay& L, int lognl, const LineTab<T>& tb) {
  if (MC == 0 && tb.n < 2) return;
  if (quarter(tb.bc)) {
    qw_pre_inverse<MAXV, T, MC>(buf, L, lognl, tb);
    fft_lines<MAXV, T, MC>(buf, L, lognl, tb);
    return;
  }
  pre_inverse<MAXV, T, MC>(buf, L, lognl, tb);
  fft_lines<MAXV, T, MC>(buf, L, lognl, tb);
}

}  // namespace cans
