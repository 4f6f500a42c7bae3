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

namespace {

template <int P, int G, int EPI>
__global__ void __launch_bounds__(256) dslash_kernel(Batch B, int out_parity, float sgn_fwd, FieldRef in, FieldRef aux,
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
    R v[24], u[18];
    // x direction
    {
      int nb = lex_of(L, (x + 1 == L.X) ? 0 : x + 1, y, z, t) >> 1;
      SIO<P>::load(inb, inn, nitems, ((long long)nb << L.lognpad) + col, v);
      GIO<G>::load(gb, L.Vh, p, 0, i, u);
      hop_term<R, false, 0>(acc, v, u, sf);
      nb = lex_of(L, (x == 0) ? L.X - 1 : x - 1, y, z, t) >> 1;
      SIO<P>::load(inb, inn, nitems, ((long long)nb << L.lognpad) + col, v);
      GIO<G>::load(gb, L.Vh, q, 0, nb, u);
      hop_term<R, true, 0>(acc, v, u, sb);
    }
    // y direction
    {
      int nb = lex_of(L, x, (y + 1 == L.Y) ? 0 : y + 1, z, t) >> 1;
      SIO<P>::load(inb, inn, nitems, ((long long)nb << L.lognpad) + col, v);
      GIO<G>::load(gb, L.Vh, p, 1, i, u);
      hop_term<R, false, 1>(acc, v, u, sf);
      nb = lex_of(L, x, (y == 0) ? L.Y - 1 : y - 1, z, t) >> 1;
      SIO<P>::load(inb, inn, nitems, ((long long)nb << L.lognpad) + col, v);
      GIO<G>::load(gb, L.Vh, q, 1, nb, u);
      hop_term<R, true, 1>(acc, v, u, sb);
    }
    // z direction
    {
      int nb = lex_of(L, x, y, (z + 1 == L.Z) ? 0 : z + 1, t) >> 1;
      SIO<P>::load(inb, inn, nitems, ((long long)nb << L.lognpad) + col, v);
      GIO<G>::load(gb, L.Vh, p, 2, i, u);
      hop_term<R, false, 2>(acc, v, u, sf);
      nb = lex_of(L, x, y, (z == 0) ? L.Z - 1 : z - 1, t) >> 1;
      SIO<P>::load(inb, inn, nitems, ((long long)nb << L.lognpad) + col, v);
      GIO<G>::load(gb, L.Vh, q, 2, nb, u);
      hop_term<R, true, 2>(acc, v, u, sb);
    }
    // t direction, with the boundary factor on hops across t = T-1 <-> 0
    {
      const R bc = (R)L.tbc;
      int nb = lex_of(L, x, y, z, (t + 1 == L.T) ? 0 : t + 1) >> 1;
      SIO<P>::load(inb, inn, nitems, ((long long)nb << L.lognpad) + col, v);
      if (t + 1 == L.T) {
#pragma unroll
        for (int m = 0; m < 24; ++m) v[m] *= bc;
      }
      GIO<G>::load(gb, L.Vh, p, 3, i, u);
      hop_term<R, false, 3>(acc, v, u, sf);
      nb = lex_of(L, x, y, z, (t == 0) ? L.T - 1 : t - 1) >> 1;
      SIO<P>::load(inb, inn, nitems, ((long long)nb << L.lognpad) + col, v);
      if (t == 0) {
#pragma unroll
        for (int m = 0; m < 24; ++m) v[m] *= bc;
      }
      GIO<G>::load(gb, L.Vh, q, 3, nb, u);
      hop_term<R, true, 3>(acc, v, u, sb);
    }
    const Epi e = ep.e[l];
    const R c = (R)e.c;
#pragma unroll
    for (int m = 0; m < 24; ++m) acc[m] *= c;
    if (EPI != EPI_PLAIN) {
      SIO<P>::load(seg_ptr<P>(aux, L), seg_norm(aux, L), nitems, j, v);
      twist_apply<R>(v, (R)e.a2, (R)e.b2);
#pragma unroll
      for (int m = 0; m < 24; ++m) acc[m] += v[m];
    }
    if (EPI == EPI_CG) {
      const R al = (R)alpha[L.rhs_base + col];
      R w[24];
      SIO<P>::load(seg_ptr<P>(cp, L), seg_norm(cp, L), nitems, j, w);   // p
      SIO<P>::load(seg_ptr<P>(cy, L), seg_norm(cy, L), nitems, j, v);   // y
#pragma unroll
      for (int m = 0; m < 24; ++m) v[m] += al * w[m];
      SIO<P>::store(seg_ptr_w<P>(cy, L), seg_norm(cy, L), nitems, j, v);
      SIO<P>::load(seg_ptr<P>(cr, L), seg_norm(cr, L), nitems, j, v);   // r
#pragma unroll
      for (int m = 0; m < 24; ++m) {
        v[m] -= al * acc[m];
        red += (double)v[m] * (double)v[m];
      }
      SIO<P>::store(seg_ptr_w<P>(cr, L), seg_norm(cr, L), nitems, j, v);
    } else {
      twist_apply<R>(acc, (R)e.a1, (R)e.b1);
      if (EPI == EPI_AUX_NORM) {
#pragma unroll
        for (int m = 0; m < 24; ++m) red += (double)acc[m] * (double)acc[m];
      }
      SIO<P>::store(seg_ptr_w<P>(out, L), seg_norm(out, L), nitems, j, acc);
    }
  }
  if (EPI == EPI_AUX_NORM || EPI == EPI_CG) block_reduce_cols(red, 1 << L.lognpad, partial);
}

template <int P, int G>
cudaError_t launch_pg(const Batch& B, int grid, int epi, float sgn, int op, FieldRef in, FieldRef aux, FieldRef out,
                      const void* g, const EpiSet& ep, const int* active, double* partial, FieldRef cr, FieldRef cy,
                      FieldRef cp, const double* alpha, cudaStream_t st) {
  switch (epi) {
    case EPI_PLAIN:
      DL_COUNT();
      dslash_kernel<P, G, EPI_PLAIN><<<grid, 256, 0, st>>>(B, op, sgn, in, aux, out, g, ep, active, partial, cr, cy, cp, alpha);
      break;
    case EPI_AUX:
      DL_COUNT();
      dslash_kernel<P, G, EPI_AUX><<<grid, 256, 0, st>>>(B, op, sgn, in, aux, out, g, ep, active, partial, cr, cy, cp, alpha);
      break;
    case EPI_AUX_NORM:
      DL_COUNT();
      dslash_kernel<P, G, EPI_AUX_NORM><<<grid, 256, 0, st>>>(B, op, sgn, in, aux, out, g, ep, active, partial, cr, cy, cp, alpha);
      break;
    case EPI_CG:
      DL_COUNT();
      dslash_kernel<P, G, EPI_CG><<<grid, 256, 0, st>>>(B, op, sgn, in, aux, out, g, ep, active, partial, cr, cy, cp, alpha);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

namespace dl {

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

cudaError_t dslash(const Batch& Bin, int prec, int grec, int epi, bool dag, int out_parity, FieldRef in, FieldRef aux,
                   FieldRef out, const GaugeSet& g, const EpiSet& ep, const int* active, double* partial, FieldRef cr,
                   FieldRef cy, FieldRef cp, const double* alpha, cudaStream_t st) {
  Batch B = Bin;
  int grid = blocks_for(B, 256);
  if (grid == 0) return cudaSuccess;
  float sgn = dag ? 1.0f : -1.0f;  // forward projector (1 + sgn gamma_mu)
  if (prec == P64) {
    if (grec != 18) return cudaErrorInvalidValue;
    return launch_pg<P64, G64R18>(B, grid, epi, sgn, out_parity, in, aux, out, g.g64, ep, active, partial, cr, cy, cp, alpha, st);
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
