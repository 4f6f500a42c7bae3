// Site-local vector kernels of the solver (BLAS-1 updates, conversions, norms,
// twist) and the per-column CG scalar kernels.  All reductions are per column
// and deterministic: block partial sums in fixed order, then one CTA per
// column sums the partials of its lattice's blocks in fixed order.
#include <algorithm>

#include "dl_internal.cuh"
#include "dl_kernels.h"

namespace {

#define ITEM_PROLOGUE                                                                     \
  const int l = find_lat(B, blockIdx.x);                                                  \
  const LatDesc& L = B.lat[l];                                                            \
  const int npad = 1 << L.lognpad;                                                        \
  const long long j = (long long)(blockIdx.x - B.blk_begin[l]) * blockDim.x + threadIdx.x; \
  const long long nitems = (long long)L.Vh * npad;                                        \
  const int col = (int)(j & (npad - 1));                                                  \
  const int gc = L.rhs_base + col;                                                        \
  const bool act = (j < nitems) && (col < L.ncol) && (mask == nullptr || mask[gc] != 0);

// dst = src (precision conversion)
template <int PD, int PS>
__global__ void copy_kernel(Batch B, FieldRef dst, FieldRef src, const int* mask) {
  ITEM_PROLOGUE
  if (!act) return;
  typename SIO<PS>::real v[24];
  SIO<PS>::load(seg_ptr<PS>(src, L), seg_norm(src, L), nitems, j, v);
  typename SIO<PD>::real w[24];
#pragma unroll
  for (int m = 0; m < 24; ++m) w[m] = (typename SIO<PD>::real)v[m];
  SIO<PD>::store(seg_ptr_w<PD>(dst, L), seg_norm(dst, L), nitems, j, w);
}

// out = a - b, the difference evaluated in a's arithmetic, stored in out's precision
template <int PO, int PA, int PB>
__global__ void diff_kernel(Batch B, FieldRef out, FieldRef a, FieldRef b) {
  const int* mask = nullptr;
  ITEM_PROLOGUE
  if (!act) return;
  typedef typename SIO<PA>::real RA;
  RA av[24];
  typename SIO<PB>::real bv[24];
  typename SIO<PO>::real ov[24];
  SIO<PA>::load(seg_ptr<PA>(a, L), seg_norm(a, L), nitems, j, av);
  SIO<PB>::load(seg_ptr<PB>(b, L), seg_norm(b, L), nitems, j, bv);
#pragma unroll
  for (int m = 0; m < 24; ++m) ov[m] = (typename SIO<PO>::real)(av[m] - (RA)bv[m]);
  SIO<PO>::store(seg_ptr_w<PO>(out, L), seg_norm(out, L), nitems, j, ov);
}

// x += y, then y = 0
template <int PH, int PL>
__global__ void accum_kernel(Batch B, FieldRef x, FieldRef y, const int* mask, int zero_y) {
  ITEM_PROLOGUE
  if (!act) return;
  typename SIO<PH>::real xv[24];
  typename SIO<PL>::real yv[24];
  SIO<PH>::load(seg_ptr<PH>(x, L), seg_norm(x, L), nitems, j, xv);
  SIO<PL>::load(seg_ptr<PL>(y, L), seg_norm(y, L), nitems, j, yv);
#pragma unroll
  for (int m = 0; m < 24; ++m) xv[m] += (typename SIO<PH>::real)yv[m];
  SIO<PH>::store(seg_ptr_w<PH>(x, L), seg_norm(x, L), nitems, j, xv);
  if (zero_y) {
#pragma unroll
    for (int m = 0; m < 24; ++m) yv[m] = 0;
    SIO<PL>::store(seg_ptr_w<PL>(y, L), seg_norm(y, L), nitems, j, yv);
  }
}

// r = b - a (same precision), partial |r|^2 per column
template <int P>
__global__ void xmy_norm_kernel(Batch B, FieldRef r, FieldRef b, FieldRef a, const int* mask, double* partial) {
  ITEM_PROLOGUE
  typename SIO<P>::real red = 0;  // per site-column in the storage arithmetic, FP64 across sites
  if (act) {
    typename SIO<P>::real bv[24], av[24];
    SIO<P>::load(seg_ptr<P>(b, L), seg_norm(b, L), nitems, j, bv);
    SIO<P>::load(seg_ptr<P>(a, L), seg_norm(a, L), nitems, j, av);
#pragma unroll
    for (int m = 0; m < 24; ++m) {
      bv[m] -= av[m];
      red += bv[m] * bv[m];
    }
    SIO<P>::store(seg_ptr_w<P>(r, L), seg_norm(r, L), nitems, j, bv);
  }
  block_reduce_cols((double)red, npad, partial, B.pstride);
}

// partial |v|^2 per column
template <int P>
__global__ void norm_kernel(Batch B, FieldRef v, const int* mask, double* partial) {
  ITEM_PROLOGUE
  typename SIO<P>::real red = 0;  // per site-column in the storage arithmetic, FP64 across sites
  if (act) {
    typename SIO<P>::real a[24];
    SIO<P>::load(seg_ptr<P>(v, L), seg_norm(v, L), nitems, j, a);
#pragma unroll
    for (int m = 0; m < 24; ++m) red += a[m] * a[m];
  }
  block_reduce_cols((double)red, npad, partial, B.pstride);
}

// p = r + beta p
template <int P>
__global__ void xpay_kernel(Batch B, FieldRef p, FieldRef r, const double* __restrict__ beta, const int* mask) {
  ITEM_PROLOGUE
  if (!act) return;
  typedef typename SIO<P>::real R;
  R rv[24], pv[24];
  const R be = (R)beta[gc];
  SIO<P>::load(seg_ptr<P>(r, L), seg_norm(r, L), nitems, j, rv);
  SIO<P>::load(seg_ptr<P>(p, L), seg_norm(p, L), nitems, j, pv);
#pragma unroll
  for (int m = 0; m < 24; ++m) pv[m] = rv[m] + be * pv[m];
  SIO<P>::store(seg_ptr_w<P>(p, L), seg_norm(p, L), nitems, j, pv);
}

// out = (a + i b gamma_5) in, (a, b) per lattice from ep.e[l].a1/b1
template <int P>
__global__ void twist_kernel(Batch B, FieldRef out, FieldRef in, EpiSet ep, const int* mask) {
  ITEM_PROLOGUE
  if (!act) return;
  typedef typename SIO<P>::real R;
  R v[24];
  SIO<P>::load(seg_ptr<P>(in, L), seg_norm(in, L), nitems, j, v);
  twist_apply<R>(v, epc<R>(ep.e[l].a1, ep.e[l].a1f, ep.e[l].a1l), epc<R>(ep.e[l].b1, ep.e[l].b1f, ep.e[l].b1l));
  SIO<P>::store(seg_ptr_w<P>(out, L), seg_norm(out, L), nitems, j, v);
}

template <int P>
__global__ void zero_kernel(Batch B, FieldRef v, const int* mask) {
  ITEM_PROLOGUE
  if (!act) return;
  typename SIO<P>::real a[24];
#pragma unroll
  for (int m = 0; m < 24; ++m) a[m] = 0;
  SIO<P>::store(seg_ptr_w<P>(v, L), seg_norm(v, L), nitems, j, a);
}

// One CTA per global column: sum the column's partials over its lattice's blocks.
__global__ void sum_partials_kernel(Batch B, const double* __restrict__ partial, double* __restrict__ out, int stride,
                                    int slot) {
  const int gc = blockIdx.x;
  int l = -1, col = 0;
  for (int k = 0; k < B.nlat; ++k)
    if (gc >= B.lat[k].rhs_base && gc < B.lat[k].rhs_base + B.lat[k].ncol) {
      l = k;
      col = gc - B.lat[k].rhs_base;
    }
  __shared__ double s[1024];
  double acc = 0.0;
  if (l >= 0)
    for (int b = B.blk_begin[l] + threadIdx.x; b < B.blk_begin[l + 1]; b += blockDim.x)
      acc += partial[(size_t)col * B.pstride + b];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0 && l >= 0) out[(size_t)slot * stride + gc] = s[0];
}

// alpha = rr / pAp for active columns
#define SV(slot) S[(slot) * DL_NCMAX + gc]
__global__ void cg_alpha_kernel(int ncols, double* S, int* active, int* flags) {
  int gc = blockIdx.x * blockDim.x + threadIdx.x;
  if (gc >= ncols || !active[gc]) return;
  double pap = SV(DL_S_PAP);
  if (!(pap > 0.0) || !isfinite(pap)) {
    flags[gc] |= DL_FLAG_BREAKDOWN;
    active[gc] = 0;
    SV(DL_S_ALPHA) = 0.0;
    return;
  }
  SV(DL_S_ALPHA) = SV(DL_S_RR) / pap;
}

// beta = rr_new / rr; convergence and reliable-update bookkeeping
__global__ void cg_beta_kernel(int ncols, double* S, int* active, int* flags, int* iters, double tol2, double delta) {
  int gc = blockIdx.x * blockDim.x + threadIdx.x;
  if (gc >= ncols || !active[gc]) return;
  double rrn = SV(DL_S_RRNEW);
  iters[gc] += 1;
  if (!isfinite(rrn)) {
    flags[gc] |= DL_FLAG_BREAKDOWN;
    active[gc] = 0;
    SV(DL_S_BETA) = 0.0;
    return;
  }
  SV(DL_S_BETA) = rrn / SV(DL_S_RR);
  SV(DL_S_RR) = rrn;
  double rn = sqrt(rrn);
  if (rn > SV(DL_S_MAXR)) SV(DL_S_MAXR) = rn;
  if (rrn <= tol2 * SV(DL_S_RR0)) {
    flags[gc] |= DL_FLAG_CONVERGED;
    active[gc] = 0;
  } else if (delta > 0.0 && rn < delta * SV(DL_S_MAXR)) {
    flags[gc] |= DL_FLAG_UPDATE;
  }
}
#undef SV

// Loop condition of the solver's graph: continue while some column is active
// and this launch has run fewer than *limit iterations, unless reliable updates
// are due: the loop stops when at least half of the active columns wait for
// one, or one has waited 16 iterations, so that updates are done in batches
// (each update applies the high-precision operator to every waiting column).
__global__ void cg_cond_kernel(int ncols, const int* __restrict__ active, const int* __restrict__ flags, int* counter,
                               const int* limit, int* wait, cudaGraphConditionalHandle h, int* cont) {
  const int gc = threadIdx.x;
  const int a = (gc < ncols) && active[gc] != 0;
  const int u = a && (flags[gc] & DL_FLAG_UPDATE) != 0;
  int w = 0;
  if (u) {
    w = wait[gc] + 1;
    wait[gc] = w;
  }
  const int n_a = __syncthreads_count(a);
  const int n_u = __syncthreads_count(u);
  const int old = __syncthreads_or(w >= 16);
  if (threadIdx.x == 0) {
    const int n = *counter + 1;
    *counter = n;
    const bool due = n_u > 0 && (2 * n_u >= n_a || old);
    const unsigned go = (n_a > 0 && !due && n < *limit) ? 1u : 0u;
    if (cont)
      *cont = (int)go;  // launched outside a graph: the host reads the decision
    else
      cudaGraphSetConditional(h, go);
  }
}

// <a, b> = sum conj(a) b over both parities of one column (single-column batch):
// grid-stride CTAs write partial[blk] (re) and partial[pstride + blk] (im); a
// second one-CTA kernel adds them in a fixed order.
template <int P>
__global__ void pdot_kernel(Batch B, FieldRef ae, FieldRef ao, FieldRef be, FieldRef bo, double* partial) {
  const LatDesc& L = B.lat[0];
  const long long nitems = (long long)L.Vh << L.lognpad;
  double re = 0.0, im = 0.0;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < 2 * nitems; q += (long long)gridDim.x * blockDim.x) {
    const bool odd = q >= nitems;
    const long long j = odd ? q - nitems : q;
    if ((int)(j & ((1 << L.lognpad) - 1)) >= L.ncol) continue;
    typedef typename SIO<P>::real R;
    R av[24], bv[24];
    const FieldRef& a = odd ? ao : ae;
    const FieldRef& b = odd ? bo : be;
    SIO<P>::load(seg_ptr<P>(a, L), seg_norm(a, L), nitems, j, av);
    SIO<P>::load(seg_ptr<P>(b, L), seg_norm(b, L), nitems, j, bv);
    R sr = 0, si = 0;  // one site in the storage arithmetic, FP64 across sites
#pragma unroll
    for (int m = 0; m < 12; ++m) {
      sr += av[2 * m] * bv[2 * m] + av[2 * m + 1] * bv[2 * m + 1];
      si += av[2 * m] * bv[2 * m + 1] - av[2 * m + 1] * bv[2 * m];
    }
    re += (double)sr;
    im += (double)si;
  }
  __shared__ double sr[32], si[32];
  for (int off = 16; off > 0; off >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, off);
    im += __shfl_xor_sync(0xffffffffu, im, off);
  }
  if ((threadIdx.x & 31) == 0) {
    sr[threadIdx.x >> 5] = re;
    si[threadIdx.x >> 5] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0, ti = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      tr += sr[w];
      ti += si[w];
    }
    partial[blockIdx.x] = tr;
    partial[(size_t)B.pstride + blockIdx.x] = ti;
  }
}

__global__ void pdot_final_kernel(const double* __restrict__ partial, int nblk, int pstride, double* out) {
  __shared__ double sr[256], si[256];
  double re = 0.0, im = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
    re += partial[b];
    im += partial[(size_t)pstride + b];
  }
  sr[threadIdx.x] = re;
  si[threadIdx.x] = im;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sr[threadIdx.x] += sr[threadIdx.x + w];
      si[threadIdx.x] += si[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sr[0];
    out[1] = si[0];
  }
}

template <int P>
__global__ void caxpy_kernel(Batch B, double ar, double ai, FieldRef x, FieldRef y) {
  const LatDesc& L = B.lat[0];
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nitems = (long long)L.Vh << L.lognpad;
  if (j >= nitems || (int)(j & ((1 << L.lognpad) - 1)) >= L.ncol) return;
  typedef typename SIO<P>::real R;
  R xv[24], yv[24];
  SIO<P>::load(seg_ptr<P>(x, L), seg_norm(x, L), nitems, j, xv);
  SIO<P>::load(seg_ptr<P>(y, L), seg_norm(y, L), nitems, j, yv);
#pragma unroll
  for (int m = 0; m < 12; ++m) {
    const R xr = xv[2 * m], xi = xv[2 * m + 1];
    yv[2 * m] += (R)ar * xr - (R)ai * xi;
    yv[2 * m + 1] += (R)ar * xi + (R)ai * xr;
  }
  SIO<P>::store(seg_ptr_w<P>(y, L), seg_norm(y, L), nitems, j, yv);
}

}  // namespace

namespace dl {

cudaError_t pdot(const Batch& B, int prec, FieldRef ae, FieldRef ao, FieldRef be, FieldRef bo, double* partial,
                 double* out, cudaStream_t st) {
  const long long items = (long long)B.lat[0].Vh << B.lat[0].lognpad;
  const int g = (int)std::min<long long>((2 * items + 255) / 256, std::min<long long>(4 * 152, B.pstride));
  if (g < 1) return cudaErrorInvalidValue;
  DL_COUNT();
  if (prec == P64) pdot_kernel<P64><<<g, 256, 0, st>>>(B, ae, ao, be, bo, partial);
  else if (prec == P32) pdot_kernel<P32><<<g, 256, 0, st>>>(B, ae, ao, be, bo, partial);
  else return cudaErrorInvalidValue;
  DL_COUNT();
  pdot_final_kernel<<<1, 256, 0, st>>>(partial, g, B.pstride, out);
  return cudaGetLastError();
}

cudaError_t caxpy(const Batch& Bin, int prec, double ar, double ai, FieldRef x, FieldRef y, cudaStream_t st) {
  Batch B = Bin;
  const int g = blocks_for(B, 256);
  if (!g) return cudaSuccess;
  DL_COUNT();
  if (prec == P64) caxpy_kernel<P64><<<g, 256, 0, st>>>(B, ar, ai, x, y);
  else if (prec == P32) caxpy_kernel<P32><<<g, 256, 0, st>>>(B, ar, ai, x, y);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t cg_cond(int ncols, const int* active, const int* flags, int* counter, const int* limit, int* wait,
                    cudaGraphConditionalHandle h, int* cont, cudaStream_t st) {
  DL_COUNT();
  cg_cond_kernel<<<1, DL_NCMAX, 0, st>>>(ncols, active, flags, counter, limit, wait, h, cont);
  return cudaGetLastError();
}

static int grid_of(Batch& B) { return blocks_for(B, 256); }

#define DISPATCH_P(prec, CALL) \
  switch (prec) {              \
    case P64: { constexpr int PP = P64; CALL; } break; \
    case P32: { constexpr int PP = P32; CALL; } break; \
    case P16: { constexpr int PP = P16; CALL; } break; \
    case PBF: { constexpr int PP = PBF; CALL; } break; \
    case PDF: { constexpr int PP = PDF; CALL; } break; \
    default: return cudaErrorInvalidValue; \
  }

cudaError_t copy(const Batch& Bin, int pd, int ps, FieldRef dst, FieldRef src, const int* mask, cudaStream_t st) {
  Batch B = Bin;
  int g = grid_of(B);
  if (!g) return cudaSuccess;
#define CP(a, b) if (pd == a && ps == b) { DL_COUNT(); copy_kernel<a, b><<<g, 256, 0, st>>>(B, dst, src, mask); return cudaGetLastError(); }
  CP(P64, P64) CP(P64, P32) CP(P64, P16) CP(P32, P64) CP(P32, P32) CP(P32, P16) CP(P16, P64) CP(P16, P32) CP(P16, P16)
  CP(PBF, P64) CP(P64, PBF) CP(PBF, P32) CP(P32, PBF) CP(PBF, PBF)
  CP(PDF, PDF) CP(PDF, P64) CP(P64, PDF) CP(PDF, P32) CP(P32, PDF) CP(PDF, P16) CP(P16, PDF)
#undef CP
  return cudaErrorInvalidValue;
}

cudaError_t accum(const Batch& Bin, int ph, int pl, FieldRef x, FieldRef y, const int* mask, int zero_y, cudaStream_t st) {
  Batch B = Bin;
  int g = grid_of(B);
  if (!g) return cudaSuccess;
#define AC(a, b) if (ph == a && pl == b) { DL_COUNT(); accum_kernel<a, b><<<g, 256, 0, st>>>(B, x, y, mask, zero_y); return cudaGetLastError(); }
  AC(P64, P64) AC(P64, P32) AC(P64, P16) AC(P32, P32) AC(P32, P16) AC(PDF, PDF) AC(PDF, P32) AC(PDF, P16)
#undef AC
  return cudaErrorInvalidValue;
}

cudaError_t xmy_norm(const Batch& Bin, int prec, FieldRef r, FieldRef b, FieldRef a, const int* mask, double* partial,
                     cudaStream_t st) {
  Batch B = Bin;
  int g = grid_of(B);
  if (!g) return cudaSuccess;
  DL_COUNT();
  DISPATCH_P(prec, (xmy_norm_kernel<PP><<<g, 256, 0, st>>>(B, r, b, a, mask, partial)));
  return cudaGetLastError();
}

cudaError_t norm2(const Batch& Bin, int prec, FieldRef v, const int* mask, double* partial, cudaStream_t st) {
  Batch B = Bin;
  int g = grid_of(B);
  if (!g) return cudaSuccess;
  DL_COUNT();
  DISPATCH_P(prec, (norm_kernel<PP><<<g, 256, 0, st>>>(B, v, mask, partial)));
  return cudaGetLastError();
}

cudaError_t xpay(const Batch& Bin, int prec, FieldRef p, FieldRef r, const double* beta, const int* mask, cudaStream_t st) {
  Batch B = Bin;
  int g = grid_of(B);
  if (!g) return cudaSuccess;
  DL_COUNT();
  DISPATCH_P(prec, (xpay_kernel<PP><<<g, 256, 0, st>>>(B, p, r, beta, mask)));
  return cudaGetLastError();
}

cudaError_t twist(const Batch& Bin, int prec, FieldRef out, FieldRef in, const EpiSet& ep, const int* mask, cudaStream_t st) {
  Batch B = Bin;
  int g = grid_of(B);
  if (!g) return cudaSuccess;
  DL_COUNT();
  DISPATCH_P(prec, (twist_kernel<PP><<<g, 256, 0, st>>>(B, out, in, ep, mask)));
  return cudaGetLastError();
}

cudaError_t zero(const Batch& Bin, int prec, FieldRef v, const int* mask, cudaStream_t st) {
  Batch B = Bin;
  int g = grid_of(B);
  if (!g) return cudaSuccess;
  DL_COUNT();
  DISPATCH_P(prec, (zero_kernel<PP><<<g, 256, 0, st>>>(B, v, mask)));
  return cudaGetLastError();
}

cudaError_t sum_partials(const Batch& Bin, const double* partial, double* out, int stride, int slot, int ncols_total,
                         cudaStream_t st) {
  Batch B = Bin;
  grid_of(B);
  if (ncols_total <= 0) return cudaSuccess;
  DL_COUNT();
  sum_partials_kernel<<<ncols_total, 1024, 0, st>>>(B, partial, out, stride, slot);
  return cudaGetLastError();
}

cudaError_t diff(const Batch& Bin, int po, int pa, int pb, FieldRef out, FieldRef a, FieldRef b, cudaStream_t st) {
  Batch B = Bin;
  const int g = grid_of(B);
  if (!g) return cudaSuccess;
  if (po == P32 && pa == PDF && pb == P32) {
    DL_COUNT();
    diff_kernel<P32, PDF, P32><<<g, 256, 0, st>>>(B, out, a, b);
    return cudaGetLastError();
  }
  if (po == P32 && pa == P64 && pb == P32) {
    DL_COUNT();
    diff_kernel<P32, P64, P32><<<g, 256, 0, st>>>(B, out, a, b);
    return cudaGetLastError();
  }
  return cudaErrorInvalidValue;
}

cudaError_t cg_alpha(int ncols, double* S, int* active, int* flags, cudaStream_t st) {
  DL_COUNT();
  cg_alpha_kernel<<<(ncols + 63) / 64, 64, 0, st>>>(ncols, S, active, flags);
  return cudaGetLastError();
}

cudaError_t cg_beta(int ncols, double* S, int* active, int* flags, int* iters, double tol2, double delta, cudaStream_t st) {
  DL_COUNT();
  cg_beta_kernel<<<(ncols + 63) / 64, 64, 0, st>>>(ncols, S, active, flags, iters, tol2, delta);
  return cudaGetLastError();
}

}  // namespace dl
