// x-passes of the mixed path on the warp-per-line engine (float work field, M = N/2 in
// {128, 256, 512}): forward transform along x fused with the double->float read of f or with the
// double-float residual of a refinement sweep, and inverse transform fused with the normalisation
// and the update of the iterate.  Same results as the CTA-wide kernels of kern_x.cu (which remain
// the path for other lengths); one warp per line, persistent CTAs, no CTA barrier inside a line.
#include <algorithm>

#include "async.cuh"
#include "plan.cuh"
#include "stencil.cuh"
#include "wline.cuh"

namespace cans {
namespace {

constexpr int XW_WARPS = 8;  // warps (lines in flight) per CTA

__device__ __forceinline__ void warp_block_accumulate(float v, double* dst) {
  __shared__ float red[XW_WARPS];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int w = 0; w < XW_WARPS; ++w) s += red[w];
    atomicAdd(dst, (double)s);
  }
}

// ---- sources of the forward pass ----
struct SrcF {  // f (double) rounded to float; accumulates sum f^2
  const double* __restrict__ f;  // line start, 16-byte aligned
  float acc;
  // called by all 32 lanes together (the first stage of a line): the rare inputs outside the integer
  // path's range (zeros, subnormal, tiny or huge values) take the hardware conversion in a
  // warp-uniform branch, so that the slow FP64-class conversion is not executed for every element
  __device__ __forceinline__ float2 pair(int n) {
    const double2 d = *reinterpret_cast<const double2*>(f + n);
    bool oka, okb;
    float a = d2f_rn_int(d.x, &oka), b = d2f_rn_int(d.y, &okb);
    if (!__all_sync(0xffffffffu, oka && okb)) {
      if (!oka) a = __double2float_rn(d.x);
      if (!okb) b = __double2float_rn(d.y);
    }
    acc = __fmaf_rn(a, a, __fmaf_rn(b, b, acc));
    return make_float2(a, b);
  }
  __device__ __forceinline__ float one(int n) {
    const float a = d2f_rn(f[n]);
    acc = __fmaf_rn(a, a, acc);
    return a;
  }
};

struct SrcDiv {  // f formed from the face velocities (DivArgs) at (n, j, k), rounded to float; sum f^2
  const DivArgs* d;
  double s;     // the divergence's scale
  size_t base;  // linear index of the line's first point
  int j, k;
  float acc;
  // called by all 32 lanes together, as SrcF::pair
  __device__ __forceinline__ float2 pair(int n) {
    const size_t c = base + n;
    const double x0 = d->at(s, c, n, j, k), x1 = d->at(s, c + 1, n + 1, j, k);
    if (d->fout != nullptr) *reinterpret_cast<double2*>(d->fout + c) = make_double2(x0, x1);
    bool oka, okb;
    float a = d2f_rn_int(x0, &oka), b = d2f_rn_int(x1, &okb);
    if (!__all_sync(0xffffffffu, oka && okb)) {
      if (!oka) a = __double2float_rn(x0);
      if (!okb) b = __double2float_rn(x1);
    }
    acc = __fmaf_rn(a, a, __fmaf_rn(b, b, acc));
    return make_float2(a, b);
  }
  __device__ __forceinline__ float one(int n) {
    const size_t c = base + n;
    const double x = d->at(s, c, n, j, k);
    if (d->fout != nullptr) d->fout[c] = x;
    const float a = d2f_rn(x);
    acc = __fmaf_rn(a, a, acc);
    return a;
  }
};

template <bool PLO>
struct SrcRes {  // r = f - L_h(Phi + Plo) at (n, j, k); accumulates sum r^2
  const double* __restrict__ f;
  const float* __restrict__ Phi;
  const float* __restrict__ Plo;
  const StencilDF* S;
  size_t base;
  int j, k;
  float acc;
  __device__ __forceinline__ float one(int n) {
    const float r = residual_point<PLO>(f, Phi, Plo, *S, base + n, n, j, k);
    acc = __fmaf_rn(r, r, acc);
    return r;
  }
  __device__ __forceinline__ float2 pair(int n) {
    const float2 r = residual_pair<PLO>(f, Phi, Plo, *S, base + n, n, j, k);
    acc = __fmaf_rn(r.x, r.x, __fmaf_rn(r.y, r.y, acc));
    return r;
  }
};

struct SrcF32 {  // float input (may be the output line itself: every value is read before any write)
  const float* s;
  __device__ __forceinline__ float2 pair(int n) { return *reinterpret_cast<const float2*>(s + n); }
  __device__ __forceinline__ float one(int n) { return s[n]; }
};

struct SnkF {
  float* __restrict__ o;  // line start, 8-byte aligned
  __device__ __forceinline__ void put(int s, float y) { o[s] = y; }
  __device__ __forceinline__ void put2(int s, float a, float b) {  // s even
    *reinterpret_cast<float2*>(o + s) = make_float2(a, b);
  }
};

// ---- source and sinks of the inverse pass ----
struct SrcSlots {
  const float* __restrict__ s;
  __device__ __forceinline__ float get(int i) { return s[i]; }
  __device__ __forceinline__ float2 get2(int i) { return *reinterpret_cast<const float2*>(s + i); }  // i even
};

// MODE 0: p = scale x (double).  1: Phi = scale x (+ dzf-weighted gauge sum).  2 / 4: (Phi, Plo) +=
// scale x.  3 / 5: p = Phi + Plo + scale x.  4 and 5 know Plo is zero.
template <int MODE>
struct SnkUpd {
  double* __restrict__ p;
  float* __restrict__ Phi;
  float* __restrict__ Plo;
  float scale;
  df gw;  // gauge weight dzf_k of the line (MODE 1)
  bool gauge;
  df gacc;
  df lacc;  // MODE 1: the lane's share of the line's sum, weighted by gw once per line
  const float* sphi;  // the line's Phi (and Plo) staged in shared memory (MODE >= 2)
  const float* splo;
  size_t base;
  // the update of one output value x at global offset o, its staged iterate values given (MODE >= 2)
  __device__ __forceinline__ float upd_with(float x, float phi, float plo, size_t o, double& pd) {
    const float d = x * scale;
    if (MODE == 5) {
      pd = f2d(phi) + f2d(d);
      return 0.f;
    }
    df s2 = two_sum(phi, d);
    s2 = fast_two_sum(s2.hi, (MODE <= 3) ? s2.lo + plo : s2.lo);
    if (MODE == 2 || MODE == 4) {
      Plo[o] = s2.lo;
      return s2.hi;
    }
    pd = df_to_double(s2);
    return 0.f;
  }
  __device__ __forceinline__ float upd(size_t o, float x, double& pd) {
    const float d = x * scale;
    if (MODE == 0) {
      pd = f2d(d);
    } else if (MODE == 1) {
      if (gauge) {
        const df s2 = two_sum(lacc.hi, d);
        lacc = df_make(s2.hi, __fadd_rn(lacc.lo, s2.lo));
      }
      return d;
    } else if (MODE == 5) {
      // Plo is zero: the exact widenings of Phi and d and one rounded FP64 add give the correctly
      // rounded Phi + d
      pd = f2d(sphi[(int)(o - base)]) + f2d(d);
    } else {
      const int n = (int)(o - base);
      df s2 = two_sum(sphi[n], d);
      s2 = fast_two_sum(s2.hi, (MODE <= 3) ? s2.lo + splo[n] : s2.lo);
      if (MODE == 2 || MODE == 4) {
        Plo[o] = s2.lo;
        return s2.hi;
      }
      pd = df_to_double(s2);
    }
    return 0.f;
  }
  __device__ __forceinline__ void one(size_t o, float x) {
    double pd = 0.0;
    const float h = upd(o, x, pd);
    if (MODE == 0 || MODE == 3 || MODE == 5)
      p[o] = pd;
    else
      Phi[o] = h;
  }
};

template <int MODE>
struct SnkLine {
  SnkUpd<MODE>* u;
  size_t base;
  __device__ __forceinline__ void one(int n, float x) { u->one(base + n, x); }
  __device__ __forceinline__ void pair(int n, float a, float b) {  // n even
    const size_t o = base + n;
    double pa = 0.0, pb = 0.0;
    float ha, hb;
    if (MODE >= 2) {
      // the staged iterate as one 8-byte pair per lane: lanes hold consecutive pairs, so a warp's
      // reads cover 256 contiguous bytes without bank conflicts
      const float2 ph = *reinterpret_cast<const float2*>(u->sphi + n);
      const float2 pl = (MODE <= 3) ? *reinterpret_cast<const float2*>(u->splo + n) : make_float2(0.f, 0.f);
      ha = u->upd_with(a, ph.x, pl.x, o, pa);
      hb = u->upd_with(b, ph.y, pl.y, o + 1, pb);
    } else {
      ha = u->upd(o, a, pa);
      hb = u->upd(o + 1, b, pb);
    }
    if (MODE == 0 || MODE == 3 || MODE == 5)
      *reinterpret_cast<double2*>(u->p + o) = make_double2(pa, pb);
    else
      *reinterpret_cast<float2*>(u->Phi + o) = make_float2(ha, hb);
  }
};

// MODE 0: f (double) -> float; 1, 2: the residual of a refinement sweep (Plo nonzero / zero);
// 3: the divergence of a channel's face velocities (dv), formed on the fly
template <int M, int BC, int MODE>
__global__ void __launch_bounds__(32 * XW_WARPS, (MODE == 0 || MODE == 3) ? 3 : 2)
    xfwd_w_kernel(const double* __restrict__ f, const float* __restrict__ Phi, const float* __restrict__ Plo,
                  float* __restrict__ dst, int nlines, LineTab<float> tb, StencilDF S, double* norm_acc,
                  DivArgs dv) {
  __shared__ float2 xbuf[XW_WARPS][M];
  constexpr int N = 2 * M;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float2* xb = xbuf[wid];
  float acc = 0.f;
  for (int line = blockIdx.x * XW_WARPS + wid; line < nlines; line += gridDim.x * XW_WARPS) {
    const size_t base = (size_t)line * N;
    SnkF snk{dst + base};
    if (MODE == 0) {
      SrcF src{f + base, 0.f};
      wl::forward<M, BC>(wl::Plain{xb}, tb, lane, src, snk);
      acc += src.acc;
    } else if (MODE == 3) {
      const int k = line / dv.ny;
      SrcDiv src{&dv, dv.scale(), base, line - k * dv.ny, k, 0.f};
      wl::forward<M, BC>(wl::Plain{xb}, tb, lane, src, snk);
      acc += src.acc;
    } else {
      const int k = line / S.n[1];
      SrcRes<MODE == 1> src{f, Phi, Plo, &S, base, line - k * S.n[1], k, 0.f};
      wl::forward<M, BC>(wl::Plain{xb}, tb, lane, src, snk);
      acc += src.acc;
    }
  }
  if (norm_acc != nullptr) warp_block_accumulate(acc, norm_acc);
}

// Forward transform of float lines, in place allowed (no restrict: in may equal out).
template <int M, int BC>
__global__ void __launch_bounds__(32 * XW_WARPS, M >= 256 ? 2 : 3) xfwd32_w_kernel(const float* in, float* out, int nlines,
                                                                    LineTab<float> tb) {
  __shared__ float2 xbuf[XW_WARPS][M];
  constexpr int N = 2 * M;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float2* xb = xbuf[wid];
  for (int line = blockIdx.x * XW_WARPS + wid; line < nlines; line += gridDim.x * XW_WARPS) {
    const size_t base = (size_t)line * N;
    SrcF32 src{in + base};
    SnkF snk{out + base};
    wl::forward<M, BC>(wl::Plain{xb}, tb, lane, src, snk);
  }
}

// number of iterate fields (Phi, Plo) an update mode reads
template <int MODE>
__host__ __device__ constexpr int upd_reads() {
  return MODE <= 1 ? 0 : (MODE <= 3 ? 2 : 1);
}

template <int M, int BC, int MODE>
__global__ void __launch_bounds__(32 * XW_WARPS, upd_reads<MODE>() == 2 ? 2 : 3)
    xinv_w_kernel(const float* __restrict__ src, double* __restrict__ p, float* __restrict__ Phi,
                  float* __restrict__ Plo, int nlines, float scale, LineTab<float> tb, const float* __restrict__ wz,
                  const float* __restrict__ wz_lo, int ny, DetSum gauge) {
  constexpr int N = 2 * M, NR = upd_reads<MODE>();
  extern __shared__ __align__(16) unsigned char xw_smem[];  // [XW_WARPS][M] float2, then [XW_WARPS][NR N] float
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float2* xb = reinterpret_cast<float2*>(xw_smem) + wid * M;
  float* stg = reinterpret_cast<float*>(xw_smem + (size_t)XW_WARPS * M * sizeof(float2)) + (size_t)wid * NR * N;
  SnkUpd<MODE> u{p, Phi, Plo, scale, df_make(0.f, 0.f), gauge.out != nullptr, df_make(0.f, 0.f), df_make(0.f, 0.f),
                 stg, stg + (NR == 2 ? N : 0), 0};
  for (int line = blockIdx.x * XW_WARPS + wid; line < nlines; line += gridDim.x * XW_WARPS) {
    const size_t base = (size_t)line * N;
    if (MODE == 1 && gauge.out != nullptr) {
      const int k = line / ny;
      u.gw = df_make(wz[k], wz_lo[k]);
    }
    if (NR > 0) {  // stage the line's iterate; the copies complete while the line is transformed
#pragma unroll
      for (int q = lane; q < N / 4; q += 32) {
        cp_async16(stg + 4 * q, Phi + base + 4 * q);
        if (NR == 2) cp_async16(stg + N + 4 * q, Plo + base + 4 * q);
      }
      cp_async_commit();
    }
    u.base = base;
    SrcSlots in{src + base};
    SnkLine<MODE> out{&u, base};
    wl::inverse<M, BC, true>(wl::Plain{xb}, tb, lane, in, out);
    if (NR > 0) __syncwarp();  // the staged iterate is read before the next line overwrites it
    if (MODE == 1 && gauge.out != nullptr) {  // the line's dzf_k-weighted share of the gauge sum
      u.gacc = df_add(u.gacc, df_mul(u.lacc, u.gw));
      u.lacc = df_make(0.f, 0.f);
    }
  }
  if (MODE == 1 && gauge.out != nullptr) det_sum_finish(block_sum_d((double)u.gacc.hi + (double)u.gacc.lo), gauge);
}

template <typename K>
int xw_grid(K kernel, int nlines) {
  int per_sm = 0, dev = 0, sms = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32 * XW_WARPS, 0);
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int need = (nlines + XW_WARPS - 1) / XW_WARPS;
  return std::max(1, std::min(need, std::max(per_sm, 1) * sms));
}

template <int M, int BC, int MODE>
cudaError_t xfwd_w(const cans_plan_s* P, const double* f, const float* Phi, const float* Plo, float* dst, double* acc,
                   cudaStream_t st, const DivArgs* dv = nullptr) {
  const int nlines = P->n[1] * P->n[2];
  auto k = xfwd_w_kernel<M, BC, MODE>;
  k<<<xw_grid(k, nlines), 32 * XW_WARPS, 0, st>>>(f, Phi, Plo, dst, nlines, P->tx_f, stencil_df(P), acc,
                                                  dv != nullptr ? *dv : DivArgs{});
  return cudaGetLastError();
}

template <int M, int BC, int MODE>
cudaError_t xinv_w(const cans_plan_s* P, const float* src, double* p, float* Phi, float* Plo, double scale,
                   double* gauge, cudaStream_t st) {
  const int nlines = P->n[1] * P->n[2];
  auto k = xinv_w_kernel<M, BC, MODE>;
  const size_t smem = (size_t)XW_WARPS * M * sizeof(float2) + (size_t)XW_WARPS * upd_reads<MODE>() * 2 * M * 4;
  cudaError_t e = set_smem((const void*)k, smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, sms = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * XW_WARPS, smem);
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::max(1, std::min((nlines + XW_WARPS - 1) / XW_WARPS, std::max(per_sm, 1) * sms));
  if ((size_t)grid > P->dsum_nslots) return cudaErrorInvalidConfiguration;
  k<<<grid, 32 * XW_WARPS, smem, st>>>(src, p, Phi, Plo, nlines, (float)scale, P->tx_f, P->dzf_f, P->dzf_flo, P->n[1],
                                        plan_sum(P, gauge));
  return cudaGetLastError();
}

template <int M, int BC>
cudaError_t xfwd32_w(const cans_plan_s* P, const float* in, float* out, cudaStream_t st) {
  const int nlines = P->n[1] * P->n[2];
  auto k = xfwd32_w_kernel<M, BC>;
  k<<<xw_grid(k, nlines), 32 * XW_WARPS, 0, st>>>(in, out, nlines, P->tx_f);
  return cudaGetLastError();
}

bool aligned16(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; }

}  // namespace

// Route a float x-pass to the warp engine when it applies; *handled says whether it did.
template <int MODE>
cudaError_t launch_xfwd_warp(const cans_plan_s* P, const double* f, const float* Phi, const float* Plo, float* dst,
                             double* acc, cudaStream_t st, bool* handled) {
  *handled = false;
  if (P->wblk || !aligned16(f) || !aligned16(dst)) return cudaSuccess;
  const int bc = P->bc[0];
  *handled = true;
#define XW_CASE(MM)                                                            \
  if (P->dx.m == MM) {                                                         \
    if (bc == BC_P) return xfwd_w<MM, BC_P, MODE>(P, f, Phi, Plo, dst, acc, st);   \
    if (bc == BC_NN) return xfwd_w<MM, BC_NN, MODE>(P, f, Phi, Plo, dst, acc, st); \
    if (bc == BC_ND) return xfwd_w<MM, BC_ND, MODE>(P, f, Phi, Plo, dst, acc, st); \
    if (bc == BC_DN) return xfwd_w<MM, BC_DN, MODE>(P, f, Phi, Plo, dst, acc, st); \
    return xfwd_w<MM, BC_DD, MODE>(P, f, Phi, Plo, dst, acc, st);                  \
  }
  XW_CASE(128)
  XW_CASE(256)
  XW_CASE(512)
#undef XW_CASE
  *handled = false;
  return cudaSuccess;
}

// the divergence source on the warp engine: periodic x lines (the channel) of the supported lengths
cudaError_t launch_xfwd_div_warp(const cans_plan_s* P, const DivArgs& d, float* dst, double* acc, cudaStream_t st,
                                 bool* handled) {
  *handled = false;
  if (P->wblk || P->bc[0] != BC_P || !aligned16(dst) || (d.fout != nullptr && !aligned16(d.fout)) ||
      !aligned16(d.u) || !aligned16(d.v) || !aligned16(d.w))
    return cudaSuccess;
  *handled = true;
  if (P->dx.m == 128) return xfwd_w<128, BC_P, 3>(P, nullptr, nullptr, nullptr, dst, acc, st, &d);
  if (P->dx.m == 256) return xfwd_w<256, BC_P, 3>(P, nullptr, nullptr, nullptr, dst, acc, st, &d);
  if (P->dx.m == 512) return xfwd_w<512, BC_P, 3>(P, nullptr, nullptr, nullptr, dst, acc, st, &d);
  *handled = false;
  return cudaSuccess;
}

template <int MODE>
cudaError_t launch_xinv_warp(const cans_plan_s* P, const float* src, double* p, float* Phi, float* Plo, double scale,
                             double* gauge, cudaStream_t st, bool* handled) {
  *handled = false;
  if (P->wblk || !aligned16(src)) return cudaSuccess;
  if ((MODE == 0 || MODE == 3 || MODE == 5) && !aligned16(p)) return cudaSuccess;
  if (upd_reads<MODE>() > 0 && !aligned16(Phi)) return cudaSuccess;
  if (upd_reads<MODE>() == 2 && !aligned16(Plo)) return cudaSuccess;
  const int bc = P->bc[0];
  *handled = true;
#define XW_CASE(MM)                                                                       \
  if (P->dx.m == MM) {                                                                    \
    if (bc == BC_P) return xinv_w<MM, BC_P, MODE>(P, src, p, Phi, Plo, scale, gauge, st);   \
    if (bc == BC_NN) return xinv_w<MM, BC_NN, MODE>(P, src, p, Phi, Plo, scale, gauge, st); \
    if (bc == BC_ND) return xinv_w<MM, BC_ND, MODE>(P, src, p, Phi, Plo, scale, gauge, st); \
    if (bc == BC_DN) return xinv_w<MM, BC_DN, MODE>(P, src, p, Phi, Plo, scale, gauge, st); \
    return xinv_w<MM, BC_DD, MODE>(P, src, p, Phi, Plo, scale, gauge, st);                  \
  }
  XW_CASE(128)
  XW_CASE(256)
  XW_CASE(512)
#undef XW_CASE
  *handled = false;
  return cudaSuccess;
}

// Residual sweep, split form: the streaming residual stencil (kern_res.cu) writes r into W, then
// this x-forward transforms W in place.  Taken whenever the x lines fit the warp engine.
bool xres_warp_ok(const cans_plan_s* P, const float* W) {
  return !P->wblk && aligned16(W) && wl::supported(P->dx.m);
}

cudaError_t launch_xfwd32_warp(const cans_plan_s* P, float* W, cudaStream_t st) {
  const int bc = P->bc[0];
#define XW_CASE(MM)                                                \
  if (P->dx.m == MM) {                                             \
    if (bc == BC_P) return xfwd32_w<MM, BC_P>(P, W, W, st);        \
    if (bc == BC_NN) return xfwd32_w<MM, BC_NN>(P, W, W, st);      \
    if (bc == BC_ND) return xfwd32_w<MM, BC_ND>(P, W, W, st);      \
    if (bc == BC_DN) return xfwd32_w<MM, BC_DN>(P, W, W, st);      \
    return xfwd32_w<MM, BC_DD>(P, W, W, st);                       \
  }
  XW_CASE(128)
  XW_CASE(256)
  XW_CASE(512)
#undef XW_CASE
  return cudaErrorInvalidValue;
}

#define XW_INST_F(MODE)                                                                                         \
  template cudaError_t launch_xfwd_warp<MODE>(const cans_plan_s*, const double*, const float*, const float*, float*, \
                                              double*, cudaStream_t, bool*);
#define XW_INST_I(MODE)                                                                                       \
  template cudaError_t launch_xinv_warp<MODE>(const cans_plan_s*, const float*, double*, float*, float*, double, \
                                              double*, cudaStream_t, bool*);
XW_INST_F(0)
XW_INST_F(1)
XW_INST_F(2)
XW_INST_I(0)
XW_INST_I(1)
XW_INST_I(2)
XW_INST_I(3)
XW_INST_I(4)
XW_INST_I(5)

}  // namespace cans
