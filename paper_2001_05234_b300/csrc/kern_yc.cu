// y-pass of the mixed path with the x-slots across the lanes (float work field, Ny = 2M with M in
// {128, 256, 512}, Nx a multiple of 16): the transform F^y of Eq. poi_reduced, forward or inverse,
// as a four-step FFT of the packed half-length line.
//
// A tile is 16 consecutive x-slots x Ny rows of one z-plane, fetched with 16-byte cp.async copies
// into shared memory (64-byte rows; rows r and r^1 trade places where bit SB of r is set, so that the
// two half-warps below always read opposite bank halves).  T = M/32 threads per x-slot work on the
// tile; thread (g, l) owns x-slot l and
//   forward: reads z_m, m = g + T q (q = 0..31) of its slot's packed line, runs a 32-point DFT over q
//            in registers, multiplies by exp(-2 pi i g ka / M), and after one exchange through the
//            tile's own buffer holds every g of its ka values, on which it runs T-point DFTs over g:
//            Z_{ka + 32 kb}.  Its ka values come in pairs (ka, 32 - ka) (thread 0: 0 and 16), so the
//            partner Z_{M-k} of the real-FFT split (and of Makhoul's twiddle for walls) is in its own
//            registers, and each output slot goes from registers straight to global memory;
//   inverse: the same steps in reverse order on conj(Z) (pairing first, T-point DFTs, twiddle,
//            exchange, 32-point DFTs), and the samples go straight to global memory.
// Quarter-wave lines (a Neumann wall paired with a Dirichlet wall) need no partner: pre-twiddle on
// the way in, post-twiddle on the way out, the same routine both ways (forward factor 2, inverse 1).
// Per element this costs one shared-memory read of the staged tile and one exchange, against the
// per-stage exchanges of a line held by one warp.  The next tile's copies are issued as soon as the
// exchange has been read and run under the rest of the current tile.
#include <algorithm>

#include "async.cuh"
#include "plan.cuh"

namespace cans {
namespace {

constexpr int YC_L = 16;  // x-slots per tile

// cos(2 pi j / 32) for 0 <= j <= 8
__host__ __device__ constexpr float yc_cq(int j) {
  return j == 0   ? 1.0f
         : j == 1 ? 0.980785280403230449126f
         : j == 2 ? 0.923879532511286756128f
         : j == 3 ? 0.831469612302545237079f
         : j == 4 ? 0.707106781186547524401f
         : j == 5 ? 0.555570233019602224743f
         : j == 6 ? 0.382683432365089771728f
         : j == 7 ? 0.195090322016128267848f
                  : 0.0f;
}
// cos(2 pi e / 32) for any integer e
__host__ __device__ constexpr float yc_cos(int e) {
  e &= 31;
  if (e > 16) e = 32 - e;
  return e <= 8 ? yc_cq(e) : -yc_cq(16 - e);
}
// x exp(-2 pi i e / 32); e is a constant once the loops around the call are unrolled
__device__ __forceinline__ float2 yc_tw(float2 x, int e) {
  e &= 31;
  if (e == 0) return x;
  if (e == 8) return make_float2(x.y, -x.x);
  if (e == 16) return make_float2(-x.x, -x.y);
  if (e == 24) return make_float2(-x.y, x.x);
  const float c = yc_cos(e), s = -yc_cos(e - 8);
  return make_float2(fmaf(x.x, c, -x.y * s), fmaf(x.x, s, x.y * c));
}

// In-register DFT (forward sign) of N = N1 N2 values, natural order in and out:
// A[k1 + N1 k2] = sum_q2 W_N^{q2 k1} W_N2^{q2 k2} sum_q1 a[N2 q1 + q2] W_N1^{q1 k1}.
template <int N1, int N2>
__device__ __forceinline__ void yc_dft2(float2* a) {
  constexpr int N = N1 * N2;
  float2 b[N];
#pragma unroll
  for (int q2 = 0; q2 < N2; ++q2) {
    float2 x[N1];
#pragma unroll
    for (int q1 = 0; q1 < N1; ++q1) x[q1] = a[N2 * q1 + q2];
    Dft<N1, float2>::run(x);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) b[k1 * N2 + q2] = yc_tw(x[k1], q2 * k1 * (32 / N));
  }
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) {
    Dft<N2, float2>::run(b + k1 * N2);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) a[k1 + N1 * k2] = b[k1 * N2 + k2];
  }
}
template <int N>
__device__ __forceinline__ void yc_dft(float2* a) {
  static_assert(N == 4 || N == 8 || N == 16 || N == 32, "DFT length");
  if constexpr (N == 4 || N == 8)
    Dft<N, float2>::run(a);
  else if constexpr (N == 16)
    yc_dft2<4, 4>(a);
  else
    yc_dft2<4, 8>(a);
}

// ka value of register block i of thread g: blocks 2s, 2s+1 hold the pair (g + T s, 32 - g - T s);
// thread 0's first pair is (0, 16), both their own partners' blocks
template <int T>
__device__ __forceinline__ int yc_ka(int g, int i) {
  const int s = i >> 1;
  if ((i & 1) == 0) return g + T * s;
  return (g == 0 && s == 0) ? 16 : 32 - g - T * s;
}

template <int M, int BC, int DIR>
__global__ void __launch_bounds__(YC_L*(M / 32), 512 / (YC_L * (M / 32)))
    yc_kernel(float* __restrict__ w, int nx, int nz, LineTab<float> tb) {
  constexpr int T = M / 32, NT = YC_L * T, N = 2 * M, NK = 32 / T;
  constexpr bool QW = (BC == BC_ND || BC == BC_DN);
  constexpr bool WALL = (BC == BC_NN || BC == BC_DD);
  // swap bit of the staged rows: what the first reads of each direction need
  constexpr int SB = WALL ? (DIR > 0 ? 2 : 0) : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* S = reinterpret_cast<float*>(smem_raw);    // staged tile: N rows x 16 floats
  float2* E = reinterpret_cast<float2*>(smem_raw);  // exchange in the same bytes: [ka][g][l]
  const int tid = threadIdx.x, l = tid & (YC_L - 1), g = tid >> 4;
  const int tiles_x = nx / YC_L, ntiles = tiles_x * nz;
  const size_t plane = (size_t)nx * N;
  const float2* __restrict__ tw = tb.tw;      // exp(-2 pi i t / M)
  const float2* __restrict__ post = tb.post;  // walls / periodic: exp(-2 pi i k / N); quarter: exp(-i pi k / N)
  const float2* __restrict__ mak = tb.mak;    // walls: exp(-i pi k / 2N); quarter: exp(-i pi (4m+1) / 4N)
  auto phys = [](int r) { return SB ? (r ^ ((r >> SB) & 1)) : r; };
  auto ld = [&](int r) { return S[phys(r) * YC_L + l]; };
  auto tile_base = [&](int t) { return w + (size_t)(t / tiles_x) * plane + (size_t)(t % tiles_x) * YC_L; };
  auto fetch = [&](int t) {
    const float* gb = tile_base(t);
#pragma unroll 4
    for (int c = tid; c < 4 * N; c += NT) {
      const int r = c >> 2, p = c & 3;
      cp_async16(S + phys(r) * YC_L + 4 * p, gb + (size_t)r * nx + 4 * p);
    }
    cp_async_commit();
  };
  auto sample_of = [](int n) { return (n < M) ? 2 * n : 2 * (N - 1 - n) + 1; };  // Makhoul order
  auto wslot = [](int s) { return BC == BC_DD ? N - 1 - s : s; };  // Dirichlet slots mirrored

  int t = blockIdx.x;
  if (t < ntiles) fetch(t);
  float2 a[32];
  for (; t < ntiles; t += gridDim.x) {
    cp_async_wait<0>();
    __syncthreads();
    float* ob = tile_base(t) + l;  // row r of this thread's slot at ob[r nx]
    auto put = [&](int r, float y) { ob[(size_t)r * nx] = y; };

    if (DIR > 0 || QW) {
      // ---- step-1 layout: z_m, m = g + T q ----
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int m = g + T * q;
        if constexpr (QW) {
          float x1 = ld(N - 1 - 2 * m);
          if (BC == BC_DN) x1 = -x1;
          a[q] = cmul(make_float2(ld(2 * m), x1), __ldg(&mak[m]));
        } else if constexpr (WALL) {
          const int n0 = sample_of(2 * m), n1 = sample_of(2 * m + 1);
          float x0 = ld(n0), x1 = ld(n1);
          if (BC == BC_DD) {  // sine transform: cosine transform of the sign-alternated input
            if (n0 & 1) x0 = -x0;
            if (n1 & 1) x1 = -x1;
          }
          a[q] = make_float2(x0, x1);
        } else {
          a[q] = make_float2(ld(2 * m), ld(2 * m + 1));
        }
      }
      yc_dft<32>(a);
#pragma unroll
      for (int ka = 1; ka < 32; ++ka) a[ka] = cmul(a[ka], __ldg(&tw[g * ka]));
      __syncthreads();  // every thread has read the staged tile
#pragma unroll
      for (int ka = 0; ka < 32; ++ka) E[(ka * T + g) * YC_L + l] = a[ka];
      __syncthreads();
#pragma unroll
      for (int i = 0; i < NK; ++i) {
        const int ka = yc_ka<T>(g, i);
#pragma unroll
        for (int gg = 0; gg < T; ++gg) a[i * T + gg] = E[(ka * T + gg) * YC_L + l];
      }
      __syncthreads();  // the buffer is free for the next tile
      if (t + (int)gridDim.x < ntiles) fetch(t + gridDim.x);
#pragma unroll
      for (int i = 0; i < NK; ++i) yc_dft<T>(a + i * T);  // a[i T + kb] = Z_{ka_i + 32 kb}

      if constexpr (QW) {
        const float F = DIR > 0 ? 2.f : 1.f;
#pragma unroll
        for (int i = 0; i < NK; ++i) {
          const int ka = yc_ka<T>(g, i);
#pragma unroll
          for (int kb = 0; kb < T; ++kb) {
            const int k = ka + 32 * kb;
            const float2 u = cmul(a[i * T + kb], __ldg(&post[k]));
            const int pa = (BC == BC_DN) ? N - 1 - 2 * k : 2 * k, pb = (BC == BC_DN) ? 2 * k : N - 1 - 2 * k;
            put(pa, F * u.x);
            put(pb, -F * u.y);
          }
        }
      } else {
        // outputs of k and M - k from Z_k, Z_{M-k}:  V_k = E + w O, V_{M-k} = conj(E - w O), w = exp(-2 pi i k/N)
        auto out_pair = [&](float2 zk, float2 zm, int k, bool both) {
          const float2 Ev = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
          const float2 Ov = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
          const float2 wO = cmul(__ldg(&post[k]), Ov);
          const float2 vk = make_float2(Ev.x + wO.x, Ev.y + wO.y);
          const float2 vm = make_float2(Ev.x - wO.x, wO.y - Ev.y);
          if constexpr (!WALL) {
            put(2 * k, vk.x);
            put(2 * k + 1, vk.y);
            if (both) {
              put(2 * (M - k), vm.x);
              put(2 * (M - k) + 1, vm.y);
            }
          } else {
            // Makhoul: Y = 2 Re(c V), -2 Im(c V) with c = exp(-i pi k / 2N); c_{M-k} = exp(-i pi/4) conj(c_k)
            const float2 c = __ldg(&mak[k]);
            const float2 ak = cmul(c, vk);
            put(wslot(k), 2.f * ak.x);
            put(wslot(N - k), -2.f * ak.y);
            if (both) {
              const float r = 0.70710678118654752440f;
              const float2 cm = make_float2(r * (c.x - c.y), -r * (c.x + c.y));
              const float2 am = cmul(cm, vm);
              put(wslot(M - k), 2.f * am.x);
              put(wslot(M + k), -2.f * am.y);
            }
          }
        };
#pragma unroll
        for (int s = 0; s < NK / 2; ++s) {
          if (s == 0 && g == 0) {
            // ka = 0 (block 0): k = 0, the self-paired k = M/2, pairs kb <-> T - kb
            {
              const float2 z0 = a[0];
              const float v0 = z0.x + z0.y, vmx = z0.x - z0.y;
              if constexpr (!WALL) {
                put(0, v0);
                put(1, vmx);
              } else {
                put(wslot(0), 2.f * v0);
                put(wslot(M), 1.41421356237309504880f * vmx);
              }
            }
            out_pair(a[T / 2], a[T / 2], M / 2, false);
#pragma unroll
            for (int kb = 1; kb < T / 2; ++kb) out_pair(a[kb], a[T - kb], 32 * kb, true);
            // ka = 16 (block 1): pairs kb <-> T - 1 - kb
#pragma unroll
            for (int kb = 0; kb < T / 2; ++kb) out_pair(a[T + kb], a[2 * T - 1 - kb], 16 + 32 * kb, true);
          } else {
            const int ka = yc_ka<T>(g, 2 * s);
#pragma unroll
            for (int kb = 0; kb < T; ++kb)
              out_pair(a[2 * s * T + kb], a[(2 * s + 1) * T + T - 1 - kb], ka + 32 * kb, true);
          }
        }
      }
    } else {
      // ---- inverse (periodic, walls): step-2 layout first, k = ka_i + 32 kb ----
#pragma unroll
      for (int i = 0; i < NK; ++i) {
        const int ka = yc_ka<T>(g, i);
#pragma unroll
        for (int kb = 0; kb < T; ++kb) {
          const int k = ka + 32 * kb;
          if constexpr (WALL)
            a[i * T + kb] = make_float2(ld(wslot(k)), ld(wslot(k == 0 ? M : N - k)));  // k = 0: (Y_0, Y_M)
          else
            a[i * T + kb] = make_float2(ld(2 * k), ld(2 * k + 1));  // k = 0: (X_0, X_M)
        }
      }
      // conj(Z_k) and conj(Z_{M-k}) from the input pair of k and M - k
      auto in_pair = [&](float2& xa, float2& xb, int k) {
        float2 xk = xa, xm = xb;
        const float2 pk = __ldg(&post[k]);
        if constexpr (WALL) {  // V_k = conj(c_k) (Y_k, -Y_{N-k}) / 2; conj(c_{M-k}) = exp(i pi/4) c_k
          const float2 c = __ldg(&mak[k]);
          const float r = 0.70710678118654752440f;
          const float2 cm = make_float2(r * (c.x - c.y), r * (c.x + c.y));
          xk = cmul(cconj(c), make_float2(0.5f * xa.x, -0.5f * xa.y));
          xm = cmul(cm, make_float2(0.5f * xb.x, -0.5f * xb.y));
        }
        const float2 A = make_float2(xk.x + xm.x, xk.y - xm.y);
        const float2 B = make_float2(xk.x - xm.x, xk.y + xm.y);
        const float2 wB = cmul(cconj(pk), B);
        xa = make_float2(A.x - wB.y, -(A.y + wB.x));
        xb = make_float2(A.x + wB.y, A.y - wB.x);
      };
#pragma unroll
      for (int s = 0; s < NK / 2; ++s) {
        if (s == 0 && g == 0) {
          {
            float2 x0 = a[0];
            if constexpr (WALL) x0 = make_float2(0.5f * x0.x, 0.70710678118654752440f * x0.y);
            a[0] = make_float2(x0.x + x0.y, -(x0.x - x0.y));
          }
          {
            float2 xa = a[T / 2], xb = a[T / 2];
            in_pair(xa, xb, M / 2);
            a[T / 2] = xa;
          }
#pragma unroll
          for (int kb = 1; kb < T / 2; ++kb) in_pair(a[kb], a[T - kb], 32 * kb);
#pragma unroll
          for (int kb = 0; kb < T / 2; ++kb) in_pair(a[T + kb], a[2 * T - 1 - kb], 16 + 32 * kb);
        } else {
          const int ka = yc_ka<T>(g, 2 * s);
#pragma unroll
          for (int kb = 0; kb < T; ++kb) in_pair(a[2 * s * T + kb], a[(2 * s + 1) * T + T - 1 - kb], ka + 32 * kb);
        }
      }
#pragma unroll
      for (int i = 0; i < NK; ++i) {
        yc_dft<T>(a + i * T);  // over kb: a[i T + gg]
        const int ka = yc_ka<T>(g, i);
#pragma unroll
        for (int gg = 1; gg < T; ++gg) a[i * T + gg] = cmul(a[i * T + gg], __ldg(&tw[gg * ka]));
      }
      __syncthreads();  // every thread has read the staged tile
#pragma unroll
      for (int i = 0; i < NK; ++i) {
        const int ka = yc_ka<T>(g, i);
#pragma unroll
        for (int gg = 0; gg < T; ++gg) E[(ka * T + gg) * YC_L + l] = a[i * T + gg];
      }
      __syncthreads();
#pragma unroll
      for (int ka = 0; ka < 32; ++ka) a[ka] = E[(ka * T + g) * YC_L + l];
      __syncthreads();  // the buffer is free for the next tile
      if (t + (int)gridDim.x < ntiles) fetch(t + gridDim.x);
      yc_dft<32>(a);  // a[q] = conj(N x-packed) at m = g + T q
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int m = g + T * q;
        const float x0 = a[q].x, x1 = -a[q].y;
        if constexpr (WALL) {
          const int n0 = sample_of(2 * m), n1 = sample_of(2 * m + 1);
          put(n0, (BC == BC_DD && (n0 & 1)) ? -x0 : x0);
          put(n1, (BC == BC_DD && (n1 & 1)) ? -x1 : x1);
        } else {
          put(2 * m, x0);
          put(2 * m + 1, x1);
        }
      }
    }
  }
}

template <int M, int BC, int DIR>
cudaError_t yc(const cans_plan_s* P, float* w, cudaStream_t st) {
  auto k = yc_kernel<M, BC, DIR>;
  constexpr int NT = YC_L * (M / 32);
  const size_t smem = (size_t)M * 128;
  cudaError_t e = set_smem((const void*)k, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, smem);
  const int ntiles = (P->n[0] / YC_L) * P->n[2];
  k<<<std::max(1, std::min(ntiles, std::max(per_sm, 1) * sms)), NT, smem, st>>>(w, P->n[0], P->n[2], P->ty_f);
  return cudaGetLastError();
}

}  // namespace

template <int DIR>
cudaError_t launch_y_cols(const cans_plan_s* P, float* w, cudaStream_t st, bool* handled) {
  *handled = false;
  if (P->wblk || P->n[0] % YC_L != 0 || (reinterpret_cast<uintptr_t>(w) & 15) || P->n[1] != 2 * P->dy.m) return cudaSuccess;
  const int bc = P->bc[1];
  *handled = true;
#define YC_CASE(MM)                                       \
  if (P->dy.m == MM) {                                    \
    if (bc == BC_P) return yc<MM, BC_P, DIR>(P, w, st);   \
    if (bc == BC_NN) return yc<MM, BC_NN, DIR>(P, w, st); \
    if (bc == BC_ND) return yc<MM, BC_ND, DIR>(P, w, st); \
    if (bc == BC_DN) return yc<MM, BC_DN, DIR>(P, w, st); \
    return yc<MM, BC_DD, DIR>(P, w, st);                  \
  }
  YC_CASE(128)
  YC_CASE(256)
  YC_CASE(512)
#undef YC_CASE
  *handled = false;
  return cudaSuccess;
}

template cudaError_t launch_y_cols<1>(const cans_plan_s*, float*, cudaStream_t, bool*);
template cudaError_t launch_y_cols<-1>(const cans_plan_s*, float*, cudaStream_t, bool*);

}  // namespace cans
