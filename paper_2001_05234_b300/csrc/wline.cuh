// Warp-per-line real transforms of contiguous lines (the operator F^x of Eq. poi_reduced and its
// inverse: real DFT for periodic, DCT-II/DST-II for Neumann/Dirichlet walls).
//
// One warp (or a group of G warps, then "lane" is the index 0..32G-1 inside the group and the
// syncs are a named barrier of the group) owns one line of N = 2M reals, M = 32 G V with V = 4, 8
// or 16 complex values per lane.
// The line is packed into M complex numbers z_m = (v_2m, v_2m+1) of the (Makhoul-permuted,
// sign-alternated for Dirichlet) sequence v and transformed by a Stockham FFT whose radices all
// divide V, so every butterfly of a stage sits in one lane's registers: lane p always holds the
// elements m = p + 32 t, t = 0..V-1, on entry to a stage, and the elements a stage produces travel
// to their next owner through a per-warp shared buffer (__syncwarp only, no CTA barrier).  Each
// exchange uses its own XOR swizzle: after a stage of stride Ns < 16 and radix R, bits
// [log2 Ns, 4) of the element index are flipped by the group index above log2(R Ns), which makes
// every exchange free of bank conflicts (8-byte accesses; checked for M = 128, 256, 512).
//
// The first stage reads its inputs through the caller's source and the post-processing of the
// real-FFT split (V_k = E_k + exp(-2 pi i k/N) O_k, then Makhoul's quarter-wave twiddle for the
// cosine/sine transforms) writes each output slot through the caller's sink, so a pass never
// stages whole lines in shared memory.  Output slot order: periodic -- slot 0 = X_0, slot 1 = X_M,
// slots 2k, 2k+1 = Re, Im X_k (1 <= k < M); Neumann -- slot k = Y_k; Dirichlet -- slot N-1-k = Y_k
// (the order of the plan's eigenvalues).
#pragma once
#include <cuda_runtime.h>

#include "lines.cuh"

namespace cans {
namespace wl {

// radix schedule for a line held by G warps (V = M / (32 G) values per lane): powers of two only,
// each radix (8, 4 or 2, largest first) dividing V
__host__ __device__ constexpr int radix(int M, int s, int G = 1) {
  int x = M, V = M / (32 * G);
  for (int i = 0;; ++i) {
    int r = (x % 8 == 0 && V % 8 == 0) ? 8 : (x % 4 == 0 && V % 4 == 0) ? 4 : 2;
    if (i == s) return r;
    x /= r;
  }
}
__host__ __device__ constexpr int nstages(int M, int G = 1) {
  int x = M, n = 0;
  while (x > 1) {
    x /= radix(M, n, G);
    ++n;
  }
  return n;
}
__host__ __device__ constexpr int stride(int M, int s, int G = 1) {
  int p = 1;
  for (int i = 0; i < s; ++i) p *= radix(M, i, G);
  return p;
}

// per-stage twiddle table of the schedule (LineTab::wst): stage S >= 1 holds (R-1) x Ns entries,
// entry (r-1) Ns + k = exp(-2 pi i k r / (R Ns)), stages one after another
__host__ __device__ constexpr int wst_offset(int M, int S, int G = 1) {
  int o = 0;
  for (int s = 1; s < S; ++s) o += (radix(M, s, G) - 1) * stride(M, s, G);
  return o;
}
__host__ __device__ constexpr int wst_size(int M, int G = 1) { return wst_offset(M, nstages(M, G), G); }

// synchronisation of the G warps that share a line: __syncwarp, or named barrier `bar` of 32 G threads
template <int G>
__device__ __forceinline__ void gsync(int bar) {
  if (G == 1)
    __syncwarp();
  else
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "n"(32 * G) : "memory");
}
__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x / 2); }
__host__ __device__ constexpr bool supported(int M) { return M == 128 || M == 256 || M == 512; }

// position of element m in the exchange that follows a stage of stride Ns and radix R
template <int Ns, int R>
__device__ __forceinline__ int xpos(int m) {
  if (Ns >= 16) return m;
  return m ^ (((m >> ilog2c(R * Ns)) & (16 / Ns - 1)) << ilog2c(Ns));
}

__device__ __forceinline__ float2 ld_tw(const float2* __restrict__ t, int i) { return __ldg(&t[i]); }

// Exchange buffer of M contiguous float2 cells.
struct Plain {
  float2* p;
  __device__ __forceinline__ float2& operator[](int i) const { return p[i]; }
};

// One Stockham stage on the lane's registers.  Exchange (all but the last stage): the outputs are
// written to xb at their swizzled positions and read back in the lane-p-owns-m=p+32t order.
template <int M, int S, int G, typename XB>
__device__ __forceinline__ void stage(float2 (&v)[M / (32 * G)], const XB& xb, const float2* __restrict__ wst,
                                      int lane, int bar) {
  constexpr int L = 32 * G;  // lanes per line
  constexpr int V = M / L, R = radix(M, S, G), Ns = stride(M, S, G), Q = V / R, NST = nstages(M, G);
  constexpr int OFF = wst_offset(M, S, G);  // this stage's block of the twiddle table
  static_assert(V % R == 0, "radix must divide the values per lane");
  static_assert(G == 1, "the plan builds the stage twiddle table for one warp per line");
  float2 w[R];
  if (Ns > 1 && Ns <= L) {  // k = lane mod Ns for every butterfly of the lane
    const int k = lane & (Ns - 1);
#pragma unroll
    for (int r = 1; r < R; ++r) w[r] = ld_tw(wst, OFF + (r - 1) * Ns + k);
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    float2 x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = v[q + Q * r];
    const int j = lane + L * q;
    const int k = j & (Ns - 1);
    if (Ns > L) {
#pragma unroll
      for (int r = 1; r < R; ++r) w[r] = ld_tw(wst, OFF + (r - 1) * Ns + k);
    }
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) x[r] = cmul(x[r], w[r]);
    }
    Dft<R, float2>::run(x);
    if (S < NST - 1) {
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) xb[xpos<Ns, R>(base + r * Ns)] = x[r];
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) v[q + Q * r] = x[r];
    }
  }
  if (S < NST - 1) {
    gsync<G>(bar);
#pragma unroll
    for (int t = 0; t < V; ++t) v[t] = xb[xpos<Ns, R>(lane + L * t)];
    gsync<G>(bar);
  }
}

template <int M, int S, int NST, int G>
struct Stages {
  template <typename XB>
  static __device__ __forceinline__ void run(float2 (&v)[M / (32 * G)], const XB& xb, const float2* wst, int lane,
                                             int bar) {
    stage<M, S, G>(v, xb, wst, lane, bar);
    Stages<M, S + 1, NST, G>::run(v, xb, wst, lane, bar);
  }
};
template <int M, int NST, int G>
struct Stages<M, NST, NST, G> {
  template <typename XB>
  static __device__ __forceinline__ void run(float2 (&)[M / (32 * G)], const XB&, const float2*, int, int) {}
};

// sample index of position n of the permuted sequence v (identity for periodic lines)
template <int BC, int N>
__device__ __forceinline__ int sample_of(int n) {
  if (BC == BC_P) return n;
  return (n < N / 2) ? 2 * n : 2 * (N - 1 - n) + 1;
}

// output slots of k: periodic (2k, 2k+1) (k = 0: X_0 and X_M in slots 0, 1), one aligned pair;
// Neumann (0, M) / (k, N-k); Dirichlet the Neumann slots s mirrored to N-1-s
template <int BC, int M, typename Snk>
__device__ __forceinline__ void put_pair(Snk& snk, int k, float o0, float o1) {
  constexpr int N = 2 * M;
  if (BC == BC_P) {
    snk.put2(2 * k, o0, o1);
  } else {
    const int s0 = k, s1 = (k == 0) ? M : N - k;
    snk.put(BC == BC_DD ? N - 1 - s0 : s0, o0);
    snk.put(BC == BC_DD ? N - 1 - s1 : s1, o1);
  }
}

// Quarter-wave line (a Neumann wall paired with a Dirichlet wall; the direction's tables hold the
// pre-twiddle exp(-i pi (4m+1)/4N) in mak and the post-twiddle exp(-i pi k/N) in post): z_m =
// (x_2m + i x_{N-1-2m}) times the pre-twiddle (sine lines: the odd sample negated), the stages, then
// u_k = Z_k times the post-twiddle gives F Re u_k and -F Im u_k at positions 2k and N-1-2k (sine
// lines: swapped).  The forward transform (DCT-IV / DST-IV) has F = 2; as both are their own
// inverses up to 2N, the inverse (times N) is the same line with F = 1 -- get/put read input
// positions and write output positions in either direction.  No partner pairing is needed.
template <int M, int BC, bool ALIAS, bool WAIT_ASYNC, int G, typename XB, typename Get, typename Put>
__device__ __forceinline__ void quarter_line(const XB& xb, const LineTab<float>& tb, int lane, float F, Get get,
                                             Put put, int bar) {
  constexpr int L = 32 * G, V = M / L, N = 2 * M;
  float2 v[V];
#pragma unroll
  for (int t = 0; t < V; ++t) {
    const int m = lane + L * t;
    const float a = get(2 * m);
    float b = get(N - 1 - 2 * m);
    if (BC == BC_DN) b = -b;  // N - 1 - 2m is odd
    v[t] = cmul(make_float2(a, b), ld_tw(tb.mak, m));
  }
  if (ALIAS) gsync<G>(bar);  // every lane has its inputs before the buffer is overwritten
  Stages<M, 0, nstages(M, G), G>::run(v, xb, tb.wst, lane, bar);
  if (WAIT_ASYNC) {  // the sink reads data the caller staged with cp.async before the line began
    asm volatile("cp.async.wait_all;" ::: "memory");
    gsync<G>(bar);
  }
#pragma unroll
  for (int t = 0; t < V; ++t) {
    const int k = lane + L * t;
    const float2 u = cmul(v[t], ld_tw(tb.post, k));
    const int pa = (BC == BC_DN) ? N - 1 - 2 * k : 2 * k, pb = (BC == BC_DN) ? 2 * k : N - 1 - 2 * k;
    put(pa, F * u.x);
    put(pb, -F * u.y);
  }
  gsync<G>(bar);
}

// Forward transform of one line.
//   src.pair(n) -> float2 (x_n, x_n+1), n even (periodic lines);  src.one(n) -> x_n (walls).
//   snk.put(s, y) stores output slot s.
// PARTNER_SHFL: take Z_{M-k} from lane 32 - p, register V-1-t by warp shuffle (lane 0 pairs within
// its own registers) instead of through the exchange buffer -- fewer shared-memory operations, all of
// v[] live through the post-processing (for callers with registers to spare); the sink may then
// write the exchange buffer directly.
template <int M, int BC, bool ALIAS = false, int G = 1, bool PARTNER_SHFL = false, typename XB, typename Src,
          typename Snk>
__device__ __forceinline__ void forward(const XB& xb, const LineTab<float>& tb, int lane, Src& src, Snk& snk,
                                        int bar = 0) {
  if constexpr (BC == BC_ND || BC == BC_DN) {
    quarter_line<M, BC, ALIAS || PARTNER_SHFL, false, G>(
        xb, tb, lane, 2.f, [&](int n) { return src.one(n); }, [&](int s, float y) { snk.put(s, y); }, bar);
    return;
  }
  constexpr int L = 32 * G, V = M / L, N = 2 * M;
  float2 v[V];
#pragma unroll
  for (int t = 0; t < V; ++t) {
    const int m = lane + L * t;
    if (BC == BC_P) {
      v[t] = src.pair(2 * m);
    } else {
      const int n0 = sample_of<BC, N>(2 * m), n1 = sample_of<BC, N>(2 * m + 1);
      float a = src.one(n0), b = src.one(n1);
      if (BC == BC_DD) {  // sine transform: cosine transform of the sign-alternated input
        if (n0 & 1) a = -a;
        if (n1 & 1) b = -b;
      }
      v[t] = make_float2(a, b);
    }
  }
  static_assert(!PARTNER_SHFL || G == 1, "shuffled partners need one warp per line");
  if (ALIAS || PARTNER_SHFL) gsync<G>(bar);  // every lane has its inputs before the buffer is overwritten
  Stages<M, 0, nstages(M, G), G>::run(v, xb, tb.wst, lane, bar);
  // v[t] = Z_k, k = lane + L t.  Partner Z_{M-k}: through the exchange buffer, or by shuffle.
  if (!PARTNER_SHFL) {
#pragma unroll
    for (int t = 0; t < V; ++t) xb[lane + L * t] = v[t];
    gsync<G>(bar);
  }
  const int src_lane = (32 - lane) & 31;
#pragma unroll
  for (int t = 0; t < V; ++t) {
    const int k = lane + L * t;
    const float2 zk = v[t];
    float2 zsh = zk;
    if (PARTNER_SHFL) {
      zsh.x = __shfl_sync(0xffffffffu, v[V - 1 - t].x, src_lane);
      zsh.y = __shfl_sync(0xffffffffu, v[V - 1 - t].y, src_lane);
      if (lane == 0) zsh = v[(V - t) % V];
    }
    float o0, o1;  // the two output values of k (slots below)
    if (k == 0) {
      const float v0 = zk.x + zk.y, vm = zk.x - zk.y;
      o0 = (BC == BC_P) ? v0 : 2.f * v0;
      o1 = (BC == BC_P) ? vm : 1.41421356237309504880f * vm;
    } else {
      const float2 zm = PARTNER_SHFL ? zsh : xb[M - k];
      float2 E, O;
      E.x = 0.5f * (zk.x + zm.x);
      E.y = 0.5f * (zk.y - zm.y);
      O.x = 0.5f * (zk.y + zm.y);
      O.y = -0.5f * (zk.x - zm.x);
      const float2 wO = cmul(ld_tw(tb.post, k), O);
      const float2 vk = make_float2(E.x + wO.x, E.y + wO.y);
      if (BC == BC_P) {
        o0 = vk.x;
        o1 = vk.y;
      } else {
        const float2 a = cmul(ld_tw(tb.mak, k), vk);
        o0 = 2.f * a.x;
        o1 = -2.f * a.y;
      }
    }
    if (ALIAS && !PARTNER_SHFL) {
      v[t] = make_float2(o0, o1);  // written after every lane has read its partners
    } else {
      put_pair<BC, M>(snk, k, o0, o1);
    }
  }
  gsync<G>(bar);
  if (ALIAS && !PARTNER_SHFL) {
#pragma unroll
    for (int t = 0; t < V; ++t) put_pair<BC, M>(snk, lane + L * t, v[t].x, v[t].y);
    gsync<G>(bar);
  }
}

// Inverse transform of one line (times N).
//   src.get(s) -> input slot s.   snk.pair(n, x_n, x_n+1) (periodic) or snk.one(n, x_n) (walls).
// Z_k from X_k and its partner X_{M-k} (k > 0): conj(A + i exp(2 pi i k/N) B), A = X_k + conj X_{M-k},
// B = X_k - conj X_{M-k}
__device__ __forceinline__ float2 pre_pair(float2 xk, float2 xm, float2 post_k) {
  const float2 A = make_float2(xk.x + xm.x, xk.y - xm.y);
  const float2 B = make_float2(xk.x - xm.x, xk.y + xm.y);
  const float2 wB = cmul(cconj(post_k), B);
  return cconj(make_float2(A.x - wB.y, A.y + wB.x));
}

// PARTNER_SHFL: X_{M-k} by warp shuffle (register pairs t, V-1-t per step; lane 0's partners are
// its own registers, copied first) instead of through the exchange buffer.
template <int M, int BC, bool WAIT_ASYNC = false, int G = 1, bool PARTNER_SHFL = false, typename XB, typename Src,
          typename Snk>
__device__ __forceinline__ void inverse(const XB& xb, const LineTab<float>& tb, int lane, Src& src, Snk& snk,
                                        int bar = 0) {
  if constexpr (BC == BC_ND || BC == BC_DN) {
    quarter_line<M, BC, true, WAIT_ASYNC, G>(
        xb, tb, lane, 1.f, [&](int s) { return src.get(s); }, [&](int n, float y) { snk.one(n, y); }, bar);
    return;
  }
  constexpr int L = 32 * G, V = M / L, N = 2 * M;
  static_assert(!PARTNER_SHFL || G == 1, "shuffled partners need one warp per line");
  float2 v[V];
  // X_k (periodic) or V_k = W^-k (Y_k - i Y_N-k)/2 (walls) for the lane's k = lane + L t
#pragma unroll
  for (int t = 0; t < V; ++t) {
    const int k = lane + L * t;
    if (BC == BC_P) {
      v[t] = src.get2(2 * k);  // (X_0, X_M) for k = 0
    } else {
      const int s0 = (BC == BC_DD) ? N - 1 : 0;
      if (k == 0) {
        v[t] = make_float2(0.5f * src.get(s0), 0.70710678118654752440f * src.get(BC == BC_DD ? N - 1 - M : M));
      } else {
        const float a = src.get(BC == BC_DD ? N - 1 - k : k), b = src.get(BC == BC_DD ? k - 1 : N - k);
        v[t] = cmul(cconj(ld_tw(tb.mak, k)), make_float2(0.5f * a, -0.5f * b));
      }
    }
  }
  // k = 0 holds (X_0, X_M) packed as real parts; every other k needs X_{M-k} from its partner
  gsync<G>(bar);  // (the source may be the exchange buffer itself)
  if (PARTNER_SHFL) {
    const int src_lane = (32 - lane) & 31;
    float2 own[V];  // lane 0: partner of register t is its own register (V - t) mod V
#pragma unroll
    for (int t = 0; t < V; ++t) own[t] = v[(V - t) % V];
#pragma unroll
    for (int t = 0; t < (V + 1) / 2; ++t) {
      const int t2 = V - 1 - t;
      float2 m1, m2;  // partners of registers t and t2: the partner lane's registers t2 and t
      m1.x = __shfl_sync(0xffffffffu, v[t2].x, src_lane);
      m1.y = __shfl_sync(0xffffffffu, v[t2].y, src_lane);
      m2.x = __shfl_sync(0xffffffffu, v[t].x, src_lane);
      m2.y = __shfl_sync(0xffffffffu, v[t].y, src_lane);
      if (lane == 0) {
        m1 = own[t];
        m2 = own[t2];
      }
      const int k1 = lane + L * t, k2 = lane + L * t2;
      const float2 z1 = (k1 == 0) ? cconj(make_float2(v[t].x + v[t].y, v[t].x - v[t].y))
                                  : pre_pair(v[t], m1, ld_tw(tb.post, k1));
      const float2 z2 = pre_pair(v[t2], m2, ld_tw(tb.post, k2));  // k2 >= L (V > 1): never 0
      v[t] = z1;
      if (t2 != t) v[t2] = z2;
    }
  } else {
#pragma unroll
    for (int t = 0; t < V; ++t) xb[lane + L * t] = v[t];
    gsync<G>(bar);
#pragma unroll
    for (int t = 0; t < V; ++t) {
      const int k = lane + L * t;
      const float2 xk = v[t];
      if (k == 0)
        v[t] = cconj(make_float2(xk.x + xk.y, xk.x - xk.y));
      else
        v[t] = pre_pair(xk, xb[M - k], ld_tw(tb.post, k));
    }
  }
  gsync<G>(bar);
  Stages<M, 0, nstages(M, G), G>::run(v, xb, tb.wst, lane, bar);
  if (WAIT_ASYNC) {  // the sink reads data the caller staged with cp.async before the line began
    asm volatile("cp.async.wait_all;" ::: "memory");
    gsync<G>(bar);
  }
  // v[t] = conj(N x-packed) at m = lane + L t: samples 2m, 2m+1 of the permuted sequence
#pragma unroll
  for (int t = 0; t < V; ++t) {
    const int m = lane + L * t;
    const float a = v[t].x, b = -v[t].y;
    if (BC == BC_P) {
      snk.pair(2 * m, a, b);
    } else {
      const int n0 = sample_of<BC, N>(2 * m), n1 = sample_of<BC, N>(2 * m + 1);
      snk.one(n0, (BC == BC_DD && (n0 & 1)) ? -a : a);
      snk.one(n1, (BC == BC_DD && (n1 & 1)) ? -b : b);
    }
  }
}

}  // namespace wl
}  // namespace cans
