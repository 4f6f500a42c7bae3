// Wilson hopping stencil with the twisted-mass site terms fused (App. A: "all
// local operators are merged into dslash kernels").
//
// One thread per (site, column) of the output parity; columns of one site are
// adjacent threads, so a link is fetched once per warp and broadcast to every
// right-hand side that uses it.  Per direction the neighbour spinor is spin
// projected to a half spinor (2 spins x 3 colours) before the SU(3) multiply.
//
// Epilogues (T = a + i b gamma_5, per lattice):
//   EPI_PLAIN     out = T1 (c D in)
//   EPI_AUX       out = T1 (c D in + T2 aux)
//   EPI_AUX_NORM  as EPI_AUX, plus per-column |out|^2 partial sums
//   EPI_CG        Ap = c D in + T2 aux (T1 = 1) stays in registers, then the CG
//                 update r -= alpha Ap, y += alpha p and per-column |r|^2
#include "dl_internal.cuh"
#include "dl_pair.cuh"

#include <map>
#include <vector>
#include <mutex>
#include <utility>

namespace {

// Epilogue shared by both thread mappings: acc holds D in (not yet scaled).
template <int P, int EPI, typename R>
__device__ __forceinline__ double epilogue(R acc[24], const Epi& e, const LatDesc& L, long long nitems, long long j,
                                           int col, const FieldRef& aux, const FieldRef& out, const FieldRef& cr,
                                           const FieldRef& cy, const FieldRef& cp, const double* alpha) {
  R red = 0;  // this site-column's |.|^2 in R; the sums over sites are FP64
  const R c = epc<R>(e.c, e.cf, e.cl);
#pragma unroll
  for (int m = 0; m < 24; ++m) acc[m] *= c;
  R v[24];
  if (EPI != EPI_PLAIN) {
    SIO<P>::load(seg_ptr<P>(aux, L), seg_norm(aux, L), nitems, j, v);
    twist_apply<R>(v, epc<R>(e.a2, e.a2f, e.a2l), epc<R>(e.b2, e.b2f, e.b2l));
#pragma unroll
    for (int m = 0; m < 24; ++m) acc[m] += v[m];
  }
  if (EPI == EPI_CG) {
    const R al = (R)alpha[L.rhs_base + col];
    SIO<P>::load(seg_ptr<P>(cr, L), seg_norm(cr, L), nitems, j, v);  // r
#pragma unroll
    for (int m = 0; m < 24; ++m) {
      v[m] -= al * acc[m];
      red += v[m] * v[m];
    }
    SIO<P>::store(seg_ptr_w<P>(cr, L), seg_norm(cr, L), nitems, j, v);
    SIO<P>::load(seg_ptr<P>(cp, L), seg_norm(cp, L), nitems, j, acc);  // p (Ap no longer needed)
    SIO<P>::load(seg_ptr<P>(cy, L), seg_norm(cy, L), nitems, j, v);    // y
#pragma unroll
    for (int m = 0; m < 24; ++m) v[m] += al * acc[m];
    SIO<P>::store(seg_ptr_w<P>(cy, L), seg_norm(cy, L), nitems, j, v);
  } else {
    twist_apply<R>(acc, epc<R>(e.a1, e.a1f, e.a1l), epc<R>(e.b1, e.b1f, e.b1l));
    if (EPI == EPI_AUX_NORM) {
#pragma unroll
      for (int m = 0; m < 24; ++m) red += acc[m] * acc[m];
    }
    SIO<P>::store(seg_ptr_w<P>(out, L), seg_norm(out, L), nitems, j, acc);
  }
  return (double)red;
}

// Neighbour of site (x,y,z,t) along direction d = 2 mu + (1 if backward): its
// checkerboard index, and whether the hop crosses the time boundary.
__device__ __forceinline__ int neighbour(const LatDesc& L, int x, int y, int z, int t, int d, bool& crosses) {
  const int mu = d >> 1;
  const bool bwd = d & 1;
  crosses = false;
  if (mu == 0) x = bwd ? (x == 0 ? L.X - 1 : x - 1) : (x + 1 == L.X ? 0 : x + 1);
  else if (mu == 1) y = bwd ? (y == 0 ? L.Y - 1 : y - 1) : (y + 1 == L.Y ? 0 : y + 1);
  else if (mu == 2) z = bwd ? (z == 0 ? L.Z - 1 : z - 1) : (z + 1 == L.Z ? 0 : z + 1);
  else {
    crosses = bwd ? (t == 0) : (t + 1 == L.T);
    t = bwd ? (t == 0 ? L.T - 1 : t - 1) : (t + 1 == L.T ? 0 : t + 1);
  }
  return lex_of(L, x, y, z, t) >> 1;
}

// Staged mapping (npad >= 4): a CTA of 256 threads covers S = 256 / npad sites.
// Phase A: 8 S threads each load and reconstruct one link (with the boundary
// sign folded in) and the neighbour index into shared memory.  Phase B: thread
// (site, column) applies the eight hops reading links from shared memory
// (broadcast to the columns of a site) and the neighbour spinors from global memory.
#ifndef DL_MINB
#define DL_MINB 4  // resident CTAs per SM the staged stencil is compiled for (best of 2, 3, 4 measured)
#endif

#ifndef DL_MINB_HI
#define DL_MINB_HI 2  // the same for the FP64 and double-float kernels (twice the registers per value)
#endif

template <int P, int G, int EPI>
__global__ void __launch_bounds__(256, (P == P64 || P == PDF) ? DL_MINB_HI : DL_MINB) dslash_staged(Batch B, int out_parity, float sgn_fwd, FieldRef in,
                                                          FieldRef aux, FieldRef out, const void* __restrict__ gbase,
                                                          EpiSet ep, const int* __restrict__ active,
                                                          double* __restrict__ partial, FieldRef cr, FieldRef cy,
                                                          FieldRef cp, const double* __restrict__ alpha) {
  typedef typename SIO<P>::real R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int l = find_lat(B, blockIdx.x);
  const LatDesc& L = B.lat[l];
  const int lg = L.lognpad;
  const int S = 256 >> lg;
  const long long item0 = (long long)(blockIdx.x - B.blk_begin[l]) * 256;
  const int site0 = (int)(item0 >> lg);
  R* su = (R*)smem_raw;               // [8][S][18]
  int* snb = (int*)(su + 8 * S * 18);  // [8][S]
  const int p = out_parity, q = 1 - p;
  const void* gb = gauge_seg<G>(gbase, L);
  for (int task = threadIdx.x; task < 8 * S; task += 256) {
    const int sl = task % S, d = task / S;
    const int i = site0 + sl;
    if (i < L.Vh) {
      int x, y, z, t;
      cb_coords(L, i, p, x, y, z, t);
      bool crosses;
      const int nb = neighbour(L, x, y, z, t, d, crosses);
      R u[18];
      GIO<G>::load(gb, L.Vh, (d & 1) ? q : p, d >> 1, (d & 1) ? nb : i, u);
      const R f = crosses ? (R)L.tbc : (R)1;
      R* dst = su + (d * S + sl) * 18;
#pragma unroll
      for (int e = 0; e < 18; ++e) dst[e] = u[e] * f;
      snb[d * S + sl] = nb;
    }
  }
  __syncthreads();
  const long long nitems = (long long)L.Vh << lg;
  const long long j = item0 + threadIdx.x;
  const int col = threadIdx.x & ((1 << lg) - 1);
  const int sl = threadIdx.x >> lg;
  const bool act = (j < nitems) && (col < L.ncol) && (active == nullptr || active[L.rhs_base + col] != 0);
  double red = 0.0;
  if (act) {
    const void* inb = seg_ptr<P>(in, L);
    const float* inn = seg_norm(in, L);
    const R sf = (R)sgn_fwd, sb = -(R)sgn_fwd;
    R acc[24];
#pragma unroll
    for (int m = 0; m < 24; ++m) acc[m] = 0;
    if constexpr (std::is_same<R, dfloat>::value) {
      // one body for the eight hops (runtime direction): the code fits the instruction cache
#pragma unroll 1
      for (int d = 0; d < 8; ++d) {
        R v[24], w;
        load_hop<P>(inb, inn, nitems, ((long long)snb[d * S + sl] << lg) + col, v, w);
        hop_term_df_rt(acc, v, su + (d * S + sl) * 18, (d & 1) ? !(sgn_fwd > 0.f) : (sgn_fwd > 0.f), w.hi > 0.f,
                       d >> 1, (d & 1) != 0);
      }
    } else {
#define HOP(D, MU, BWD)                                                                                  \
    {                                                                                                    \
      R v[24], w;                                                                                        \
      load_hop<P>(inb, inn, nitems, ((long long)snb[(D) * S + sl] << lg) + col, v, w);                   \
      hop_any<R, BWD, MU>(acc, v, su + ((D) * S + sl) * 18, BWD ? sb : sf, w);                            \
    }
      HOP(0, 0, false) HOP(1, 0, true) HOP(2, 1, false) HOP(3, 1, true)
      HOP(4, 2, false) HOP(5, 2, true) HOP(6, 3, false) HOP(7, 3, true)
#undef HOP
    }
    hop_finish<R>(acc);
    red = epilogue<P, EPI, R>(acc, ep.e[l], L, nitems, j, col, aux, out, cr, cy, cp, alpha);
  }
  if (EPI == EPI_AUX_NORM || EPI == EPI_CG) block_reduce_cols(red, 1 << lg, partial, B.pstride);
}

// Two columns per thread (FP32 and 16-bit storage, npad >= 4), packed FP32x2
// arithmetic: a CTA of 128 threads covers 256 items = S = 256 / npad sites.
// Phase A stages the 8 S links of the CTA's sites in shared memory as float4
// (re, re, im, im) per entry (boundary sign folded in) with the neighbour indices;
// phase B: thread (site, column pair) applies the eight hops with both columns in
// the two lanes of every float2.
#ifndef DL_PAIR_STENCIL
#define DL_PAIR_STENCIL 1  // 0 builds the one-column staged kernel for FP32 and 16-bit too (A/B comparisons)
#endif
#ifndef DL_MINB_PAIR
#define DL_MINB_PAIR 4  // resident 128-thread CTAs per SM the pair stencil is compiled for
#endif

template <int P, int EPI>
__device__ __forceinline__ void epilogue_pair(float2 acc[24], const Epi& e, const LatDesc& L, long long nitems,
                                              long long j0, int col0, bool w0, bool w1, const FieldRef& aux,
                                              const FieldRef& out, const FieldRef& cr, const FieldRef& cy,
                                              const FieldRef& cp, const double* alpha, float2& red) {
  red = make_float2(0.f, 0.f);
  const float2 c2 = dup2(e.cf);
  float2 v[24];
  if (EPI != EPI_PLAIN) {  // acc = c acc + T2 aux
    PIO<P>::load_values(seg_ptr<P>(aux, L), seg_norm(aux, L), nitems, j0, v);
    if (e.b2f != 0.f || e.a2f != 1.f) twist_pair(v, e.a2f, e.b2f);
#pragma unroll
    for (int m = 0; m < 24; ++m) acc[m] = fma2(c2, acc[m], v[m]);
  } else {
#pragma unroll
    for (int m = 0; m < 24; ++m) acc[m] = mul2(c2, acc[m]);
  }
  if (EPI == EPI_CG) {  // acc = Ap; r -= alpha Ap, |r|^2; y += alpha p
    // a column's step size is read only when the column is active (padding columns have none)
    const float2 al = make_float2(w0 ? (float)alpha[L.rhs_base + col0] : 0.f, w1 ? (float)alpha[L.rhs_base + col0 + 1] : 0.f);
    const float2 nal = neg2(al);
    PIO<P>::load_values(seg_ptr<P>(cr, L), seg_norm(cr, L), nitems, j0, v);
#pragma unroll
    for (int m = 0; m < 24; ++m) {
      v[m] = fma2(nal, acc[m], v[m]);
      red = fma2(v[m], v[m], red);
    }
    PIO<P>::store(seg_ptr_w<P>(cr, L), seg_norm(cr, L), nitems, j0, v, w0, w1);
    PIO<P>::load_values(seg_ptr<P>(cp, L), seg_norm(cp, L), nitems, j0, acc);  // p (Ap no longer needed)
    PIO<P>::load_values(seg_ptr<P>(cy, L), seg_norm(cy, L), nitems, j0, v);    // y
#pragma unroll
    for (int m = 0; m < 24; ++m) v[m] = fma2(al, acc[m], v[m]);
    PIO<P>::store(seg_ptr_w<P>(cy, L), seg_norm(cy, L), nitems, j0, v, w0, w1);
  } else {
    if (e.b1f != 0.f || e.a1f != 1.f) twist_pair(acc, e.a1f, e.b1f);
    if (EPI == EPI_AUX_NORM) {
#pragma unroll
      for (int m = 0; m < 24; ++m) red = fma2(acc[m], acc[m], red);
    }
    PIO<P>::store(seg_ptr_w<P>(out, L), seg_norm(out, L), nitems, j0, acc, w0, w1);
  }
  if (!w0) red.x = 0.f;
  if (!w1) red.y = 0.f;
}

// SG = 0: the projector sign sgn_fwd is read at run time; SG = +-1 (16-bit storage): it is
// sgn_fwd fixed at compile time, and the spin projection runs on the biased 16-bit values
// (project_biased_pair).
template <int P, int G, int EPI, int SG>
__global__ void __launch_bounds__(128, DL_MINB_PAIR) dslash_pair(Batch B, int out_parity, float sgn_fwd, FieldRef in,
                                                                 FieldRef aux, FieldRef out,
                                                                 const void* __restrict__ gbase, EpiSet ep,
                                                                 const int* __restrict__ active,
                                                                 double* __restrict__ partial, FieldRef cr, FieldRef cy,
                                                                 FieldRef cp, const double* __restrict__ alpha) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int l = find_lat(B, blockIdx.x);
  const LatDesc& L = B.lat[l];
  const int lg = L.lognpad;
  const int S = 256 >> lg;
  const long long item0 = (long long)(blockIdx.x - B.blk_begin[l]) * 256;
  const int site0 = (int)(item0 >> lg);
  float4* su = (float4*)smem_raw;       // [8][S][9] entries (re, re, im, im)
  int* snb = (int*)(su + 8 * S * 9);    // [8][S]
  const int p = out_parity, q = 1 - p;
  const void* gb = gauge_seg<G>(gbase, L);
  for (int task = threadIdx.x; task < 8 * S; task += 128) {
    const int sl = task % S, d = task / S;
    const int i = site0 + sl;
    if (i < L.Vh) {
      int x, y, z, t;
      cb_coords(L, i, p, x, y, z, t);
      bool crosses;
      const int nb = neighbour(L, x, y, z, t, d, crosses);
      float u[18];
      GIO<G>::load(gb, L.Vh, (d & 1) ? q : p, d >> 1, (d & 1) ? nb : i, u);
      const float f = crosses ? (float)L.tbc : 1.f;
      float4* dst = su + (d * S + sl) * 9;
#pragma unroll
      for (int e = 0; e < 9; ++e) dst[e] = make_float4(u[2 * e] * f, u[2 * e] * f, u[2 * e + 1] * f, u[2 * e + 1] * f);
      snb[d * S + sl] = nb;
    }
  }
  __syncthreads();
  const long long nitems = (long long)L.Vh << lg;
  const long long j0 = item0 + 2 * threadIdx.x;
  const int col0 = (int)(j0 & ((1 << lg) - 1));
  const int sl = (int)((2 * threadIdx.x) >> lg);
  const bool in_range = j0 < nitems;
  const bool w0 = in_range && col0 < L.ncol && (active == nullptr || active[L.rhs_base + col0] != 0);
  const bool w1 = in_range && col0 + 1 < L.ncol && (active == nullptr || active[L.rhs_base + col0 + 1] != 0);
  float2 red = make_float2(0.f, 0.f);
  if (w0 || w1) {
    const void* inb = seg_ptr<P>(in, L);
    const float* inn = seg_norm(in, L);
    const float2 sf = dup2(sgn_fwd), sb = dup2(-sgn_fwd);
    float2 acc[24];
#pragma unroll
    for (int m = 0; m < 24; ++m) acc[m] = make_float2(0.f, 0.f);
#define HOP(D, MU, BWD)                                                                     \
    {                                                                                       \
      float2 v[24], w, hr[2][3], hi[2][3];                                                  \
      const long long jn = ((long long)snb[(D) * S + sl] << lg) + col0;                     \
      if constexpr (SG != 0) {                                                              \
        constexpr int SH = BWD ? -SG : SG;                                                  \
        PIO<P>::load_biased(inb, inn, nitems, jn, v, w);                                    \
        project_biased_pair<MU, SH>(v, hr, hi);                                             \
        apply_pair<MU, BWD>(acc, hr, hi, su + ((D) * S + sl) * 9, dup2((float)SH), w);     \
      } else {                                                                              \
        PIO<P>::load(inb, inn, nitems, jn, v, w);                                           \
        project_pair<MU>(v, BWD ? sb : sf, hr, hi);                                         \
        apply_pair<MU, BWD>(acc, hr, hi, su + ((D) * S + sl) * 9, BWD ? sb : sf, w);        \
      }                                                                                     \
    }
    HOP(0, 0, false) HOP(1, 0, true) HOP(2, 1, false) HOP(3, 1, true)
    HOP(4, 2, false) HOP(5, 2, true) HOP(6, 3, false) HOP(7, 3, true)
#undef HOP
    epilogue_pair<P, EPI>(acc, ep.e[l], L, nitems, j0, col0, w0, w1, aux, out, cr, cy, cp, alpha, red);
  }
  if (EPI == EPI_AUX_NORM || EPI == EPI_CG) block_reduce_pairs((double)red.x, (double)red.y, 1 << lg, partial, B.pstride);
}

// Direct mapping (npad < 4): every thread computes its own neighbours and links.
template <int P, int G, int EPI>
__global__ void __launch_bounds__(256, (P == P64 || P == PDF) ? DL_MINB_HI : 1) dslash_kernel(Batch B, int out_parity, float sgn_fwd, FieldRef in, FieldRef aux,
                                                     FieldRef out, const void* __restrict__ gbase, EpiSet ep,
                                                     const int* __restrict__ active, double* __restrict__ partial,
                                                     FieldRef cr, FieldRef cy, FieldRef cp,
                                                     const double* __restrict__ alpha) {
  typedef typename SIO<P>::real R;
  const int l = find_lat(B, blockIdx.x);
  const LatDesc& L = B.lat[l];
  const int npad = 1 << L.lognpad;
  const long long j = (long long)(blockIdx.x - B.blk_begin[l]) * blockDim.x + threadIdx.x;
  const long long nitems = (long long)L.Vh * npad;
  const int col = (int)(j & (npad - 1));
  const bool act = (j < nitems) && (col < L.ncol) && (active == nullptr || active[L.rhs_base + col] != 0);
  double red = 0.0;
  if (act) {
    const int i = (int)(j >> L.lognpad);
    const int p = out_parity, q = 1 - p;
    int x, y, z, t;
    cb_coords(L, i, p, x, y, z, t);
    const void* inb = seg_ptr<P>(in, L);
    const float* inn = seg_norm(in, L);
    const void* gb = gauge_seg<G>(gbase, L);
    const R sf = (R)sgn_fwd, sb = -(R)sgn_fwd;
    R acc[24];
#pragma unroll
    for (int m = 0; m < 24; ++m) acc[m] = 0;
    if constexpr (std::is_same<R, dfloat>::value) {
#pragma unroll 1
      for (int d = 0; d < 8; ++d) {
        bool crosses;
        const int nb = neighbour(L, x, y, z, t, d, crosses);
        R v[24], u[18], w;
        load_hop<P>(inb, inn, nitems, ((long long)nb << L.lognpad) + col, v, w);
        GIO<G>::load(gb, L.Vh, (d & 1) ? q : p, d >> 1, (d & 1) ? nb : i, u);
        const bool wpos = !(crosses && L.tbc < 0.0);
        hop_term_df_rt(acc, v, u, (d & 1) ? !(sgn_fwd > 0.f) : (sgn_fwd > 0.f), wpos, d >> 1, (d & 1) != 0);
      }
    } else {
#define HOP(D, MU, BWD)                                                                  \
    {                                                                                    \
      bool crosses;                                                                      \
      const int nb = neighbour(L, x, y, z, t, D, crosses);                               \
      R v[24], u[18], w;                                                                 \
      load_hop<P>(inb, inn, nitems, ((long long)nb << L.lognpad) + col, v, w);           \
      GIO<G>::load(gb, L.Vh, BWD ? q : p, MU, BWD ? nb : i, u);                           \
      if (crosses) w *= (R)L.tbc;                                                        \
      hop_any<R, BWD, MU>(acc, v, u, BWD ? sb : sf, w);                                   \
    }
      HOP(0, 0, false) HOP(1, 0, true) HOP(2, 1, false) HOP(3, 1, true)
      HOP(4, 2, false) HOP(5, 2, true) HOP(6, 3, false) HOP(7, 3, true)
#undef HOP
    }
    hop_finish<R>(acc);
    red = epilogue<P, EPI, R>(acc, ep.e[l], L, nitems, j, col, aux, out, cr, cy, cp, alpha);
  }
  if (EPI == EPI_AUX_NORM || EPI == EPI_CG) block_reduce_cols(red, 1 << L.lognpad, partial, B.pstride);
}

// Dynamic shared memory above the 48 KB default needs a per-device, per-kernel
// attribute; it is set (and checked) the first time a kernel runs on a device.
template <typename K>
cudaError_t ensure_smem_attr(K kernel, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> set_bytes;  // (kernel, device) -> bytes
  int dev = 0;
  DL_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_pair((const void*)kernel, dev);
  auto it = set_bytes.find(key);
  if (it != set_bytes.end() && it->second >= bytes) return cudaSuccess;
  DL_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  set_bytes[key] = bytes;
  return cudaSuccess;
}

inline bool aligned32(const FieldRef& f) { return ((uintptr_t)f.data & 31) == 0 && ((uintptr_t)f.norm & 7) == 0; }

template <int P, int G, int EPI, int SG>
cudaError_t launch_pair(const Batch& B, int grid, size_t smem, float sgn, int op, FieldRef in, FieldRef aux, FieldRef out,
                        const void* g, const EpiSet& ep, const int* active, double* partial, FieldRef cr, FieldRef cy,
                        FieldRef cp, const double* alpha, cudaStream_t st) {
  DL_CUDA_TRY(ensure_smem_attr(dslash_pair<P, G, EPI, SG>, 8 * 64 * 9 * 16 + 8 * 64 * 4));
  DL_COUNT();
  dslash_pair<P, G, EPI, SG><<<grid, 128, smem, st>>>(B, op, sgn, in, aux, out, g, ep, active, partial, cr, cy, cp, alpha);
  return cudaGetLastError();
}

template <int P, int G, int EPI>
cudaError_t launch_epi(const Batch& B, int grid, float sgn, int op, FieldRef in, FieldRef aux, FieldRef out,
                       const void* g, const EpiSet& ep, const int* active, double* partial, FieldRef cr, FieldRef cy,
                       FieldRef cp, const double* alpha, cudaStream_t st) {
  int minlg = 31;
  bool even = true;
  for (int l = 0; l < B.nlat; ++l) {
    minlg = B.lat[l].lognpad < minlg ? B.lat[l].lognpad : minlg;
    even = even && (B.lat[l].item_off & 1) == 0;
  }
  if constexpr ((P == P32 || P == P16) && DL_PAIR_STENCIL) {
    if (minlg >= 2) {
      // two columns per thread with 32-byte accesses: every field must be 32-byte aligned
      if (!even || !aligned32(in) || !aligned32(aux) || !aligned32(out) || !aligned32(cr) || !aligned32(cy) ||
          !aligned32(cp))
        return cudaErrorMisalignedAddress;
      const int S = 256 >> minlg;
      const size_t smem = (size_t)8 * S * 9 * sizeof(float4) + (size_t)8 * S * sizeof(int);
      if constexpr (P == P16) {
        if (sgn > 0.f)
          return launch_pair<P, G, EPI, 1>(B, grid, smem, sgn, op, in, aux, out, g, ep, active, partial, cr, cy, cp, alpha, st);
        return launch_pair<P, G, EPI, -1>(B, grid, smem, sgn, op, in, aux, out, g, ep, active, partial, cr, cy, cp, alpha, st);
      } else {
        return launch_pair<P, G, EPI, 0>(B, grid, smem, sgn, op, in, aux, out, g, ep, active, partial, cr, cy, cp, alpha, st);
      }
    }
  }
  if (minlg >= 2) {
    typedef typename SIO<P>::real R;
    const int S = 256 >> minlg;
    const size_t smem = (size_t)8 * S * 18 * sizeof(R) + (size_t)8 * S * sizeof(int);
    DL_CUDA_TRY(ensure_smem_attr(dslash_staged<P, G, EPI>, 8 * 64 * 18 * 8 + 8 * 64 * 4));
    DL_COUNT();
    dslash_staged<P, G, EPI><<<grid, 256, smem, st>>>(B, op, sgn, in, aux, out, g, ep, active, partial, cr, cy, cp, alpha);
  } else {
    DL_COUNT();
    dslash_kernel<P, G, EPI><<<grid, 256, 0, st>>>(B, op, sgn, in, aux, out, g, ep, active, partial, cr, cy, cp, alpha);
  }
  return cudaGetLastError();
}

template <int P, int G>
cudaError_t launch_pg(const Batch& B, int grid, int epi, float sgn, int op, FieldRef in, FieldRef aux, FieldRef out,
                      const void* g, const EpiSet& ep, const int* active, double* partial, FieldRef cr, FieldRef cy,
                      FieldRef cp, const double* alpha, cudaStream_t st) {
  switch (epi) {
    case EPI_PLAIN:
      return launch_epi<P, G, EPI_PLAIN>(B, grid, sgn, op, in, aux, out, g, ep, active, partial, cr, cy, cp, alpha, st);
    case EPI_AUX:
      return launch_epi<P, G, EPI_AUX>(B, grid, sgn, op, in, aux, out, g, ep, active, partial, cr, cy, cp, alpha, st);
    case EPI_AUX_NORM:
      return launch_epi<P, G, EPI_AUX_NORM>(B, grid, sgn, op, in, aux, out, g, ep, active, partial, cr, cy, cp, alpha, st);
    case EPI_CG:
      return launch_epi<P, G, EPI_CG>(B, grid, sgn, op, in, aux, out, g, ep, active, partial, cr, cy, cp, alpha, st);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace

namespace dl {

namespace {
struct TimedLaunch {
  cudaEvent_t e0, e1;
  int cls;
  long long items;
};
struct StencilProf {
  std::mutex mu;
  bool on = false;
  long long n[DL_SCLASSES] = {0};
  long long timed[DL_SCLASSES] = {0};
  double ms[DL_SCLASSES] = {0};
  double items[DL_SCLASSES] = {0};
  std::vector<TimedLaunch> pending;
};
StencilProf& sprof() {
  static StencilProf p;
  return p;
}
thread_local bool t_capturing = false, t_sampling = false;
thread_local StencilTally t_tally;

int stencil_class(int prec, int epi, bool dag) {
  const int slot = prec == PDF ? 0 : (prec == P32 ? 1 : (prec == P16 ? 2 : 3));
  return (slot * 4 + epi) * 2 + (dag ? 1 : 0);
}
}  // namespace

void stencil_prof_enable(bool on) {
  StencilProf& P = sprof();
  std::lock_guard<std::mutex> lk(P.mu);
  for (auto& t : P.pending) {
    cudaEventDestroy(t.e0);
    cudaEventDestroy(t.e1);
  }
  P.pending.clear();
  P.on = on;
  for (int k = 0; k < DL_SCLASSES; ++k) {
    P.n[k] = P.timed[k] = 0;
    P.ms[k] = P.items[k] = 0.0;
  }
}
void stencil_prof_sampling(bool on) { t_sampling = on; }
void stencil_capture_begin() {
  t_capturing = true;
  t_tally = StencilTally();
}
StencilTally stencil_capture_end() {
  t_capturing = false;
  return t_tally;
}
void stencil_tally_add(const StencilTally& t, long long times) {
  StencilProf& P = sprof();
  std::lock_guard<std::mutex> lk(P.mu);
  if (!P.on) return;
  for (int k = 0; k < DL_SCLASSES; ++k) P.n[k] += t.n[k] * times;
}
cudaError_t stencil_prof_read(double* out) {
  StencilProf& P = sprof();
  std::lock_guard<std::mutex> lk(P.mu);
  cudaError_t err = cudaSuccess;
  for (auto& t : P.pending) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(t.e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t.e0, t.e1);
    if (e == cudaSuccess) {
      P.timed[t.cls] += 1;
      P.ms[t.cls] += ms;
      P.items[t.cls] += (double)t.items;
    } else {
      err = e;
    }
    cudaEventDestroy(t.e0);
    cudaEventDestroy(t.e1);
  }
  P.pending.clear();
  if (out)
    for (int k = 0; k < DL_SCLASSES; ++k) {
      out[4 * k] = (double)P.n[k];
      out[4 * k + 1] = (double)P.timed[k];
      out[4 * k + 2] = P.ms[k];
      out[4 * k + 3] = P.items[k];
    }
  return err;
}

int blocks_for(Batch& B, int threads) {
  int b = 0;
  for (int l = 0; l < B.nlat; ++l) {
    B.blk_begin[l] = b;
    long long items = (long long)B.lat[l].Vh << B.lat[l].lognpad;
    b += (int)((items + threads - 1) / threads);
  }
  B.blk_begin[B.nlat] = b;
  return b;
}

static cudaError_t dslash_launch(const Batch& Bin, int prec, int grec, int epi, bool dag, int out_parity, FieldRef in,
                                 FieldRef aux, FieldRef out, const GaugeSet& g, const EpiSet& ep, const int* active,
                                 double* partial, FieldRef cr, FieldRef cy, FieldRef cp, const double* alpha,
                                 cudaStream_t st);

// Every stencil launch: counted by class (and timed with events outside capture)
// while the statistics are enabled.
cudaError_t dslash(const Batch& Bin, int prec, int grec, int epi, bool dag, int out_parity, FieldRef in, FieldRef aux,
                   FieldRef out, const GaugeSet& g, const EpiSet& ep, const int* active, double* partial, FieldRef cr,
                   FieldRef cy, FieldRef cp, const double* alpha, cudaStream_t st) {
  StencilProf& P = sprof();
  const int cls = stencil_class(prec, epi, dag);
  if (t_capturing) t_tally.n[cls] += 1;
  const bool prof = P.on && !t_capturing;
  bool started = false;  // the start event is recorded
  TimedLaunch tl{nullptr, nullptr, cls, 0};
  if (prof) {
    for (int l = 0; l < Bin.nlat; ++l) tl.items += (long long)Bin.lat[l].Vh * Bin.lat[l].ncol;
    if (cudaEventCreate(&tl.e0) == cudaSuccess && cudaEventCreate(&tl.e1) == cudaSuccess &&
        cudaEventRecord(tl.e0, st) == cudaSuccess)
      started = true;
  }
  cudaError_t e = dslash_launch(Bin, prec, grec, epi, dag, out_parity, in, aux, out, g, ep, active, partial, cr, cy, cp,
                                alpha, st);
  bool queued = false;  // the event pair now belongs to the pending list
  if (prof) {
    std::lock_guard<std::mutex> lk(P.mu);
    if (!t_sampling) P.n[cls] += 1;
    if (started && e == cudaSuccess && cudaEventRecord(tl.e1, st) == cudaSuccess) {
      P.pending.push_back(tl);
      queued = true;
    }
  }
  if (!queued) {  // release events that were created but not handed over
    if (tl.e0) cudaEventDestroy(tl.e0);
    if (tl.e1) cudaEventDestroy(tl.e1);
  }
  return e;
}

static cudaError_t dslash_launch(const Batch& Bin, int prec, int grec, int epi, bool dag, int out_parity, FieldRef in,
                                 FieldRef aux, FieldRef out, const GaugeSet& g, const EpiSet& ep, const int* active,
                                 double* partial, FieldRef cr, FieldRef cy, FieldRef cp, const double* alpha,
                                 cudaStream_t st) {
  Batch B = Bin;
  int grid = blocks_for(B, 256);
  if (grid == 0) return cudaSuccess;
  float sgn = dag ? 1.0f : -1.0f;  // forward projector (1 + sgn gamma_mu)
  if (prec == P64) {
    if (grec != 18) return cudaErrorInvalidValue;
    return launch_pg<P64, G64R18>(B, grid, epi, sgn, out_parity, in, aux, out, g.g64, ep, active, partial, cr, cy, cp, alpha, st);
  }
  if (prec == PDF) {
    if (grec != 18 || !g.gdf) return cudaErrorInvalidValue;
    return launch_pg<PDF, GDF18>(B, grid, epi, sgn, out_parity, in, aux, out, g.gdf, ep, active, partial, cr, cy, cp, alpha, st);
  }
  if (prec == P32) {
    if (grec == 12)
      return launch_pg<P32, G32R12>(B, grid, epi, sgn, out_parity, in, aux, out, g.g32, ep, active, partial, cr, cy, cp, alpha, st);
    if (grec == 8)
      return launch_pg<P32, G32R8>(B, grid, epi, sgn, out_parity, in, aux, out, g.g32, ep, active, partial, cr, cy, cp, alpha, st);
    return cudaErrorInvalidValue;
  }
  if (prec == P16) {
    if (grec == 12)
      return launch_pg<P16, G16R12>(B, grid, epi, sgn, out_parity, in, aux, out, g.g16, ep, active, partial, cr, cy, cp, alpha, st);
    if (grec == 8)
      return launch_pg<P16, G16R8>(B, grid, epi, sgn, out_parity, in, aux, out, g.g16, ep, active, partial, cr, cy, cp, alpha, st);
    return cudaErrorInvalidValue;
  }
  return cudaErrorInvalidValue;
}

}  // namespace dl
