// Loop contractions (App. A, "Contraction kernels"): per site the colour-traced
// Dirac outer product C_ab(x) = sum_c conj(xi_ac(x)) phi_bc(x) of the two
// vectors of an estimator, the covariant-derivative bilinears, and the
// momentum projection L(t, p) = sum_x exp(-i p.x) C(x, t) done as three
// separable 1-D DFT passes (x, then y, then z) over the cube of integer
// momenta, followed by the cut |n|^2 <= P.
//
// The symmetric derivative l^mu(x) = 1/4 [H(x) + H(x - mu)] with
// H(x) = xi^+(x) U_mu(x) phi(x+mu) - xi^+(x+mu) U_mu(x)^+ phi(x) is the
// four-term definition regrouped; the shift by mu becomes the phase
// (1 + exp(-i p_mu)) for spatial mu and a sum of neighbouring time slices for t.
#include "dl_internal.cuh"
#include "dl_kernels.h"
#include "dl_pair.cuh"

namespace {

enum { MODE_STANDARD = 0, MODE_ONE_END = 1, MODE_GEN = 2, MODE_HPE = 3 };

template <int P, typename R>
__device__ __forceinline__ void load_r(const FieldRef& f, const LatDesc& L, long long nitems, long long j, R v[24]) {
  typename SIO<P>::real a[24];
  SIO<P>::load(seg_ptr<P>(f, L), seg_norm(f, L), nitems, j, a);
#pragma unroll
  for (int m = 0; m < 24; ++m) v[m] = (R)a[m];
}

// (xi, phi) of an estimator at one site from s (or w) and eta, in the
// arithmetic type R (FP32 for the low-precision pipeline: no FP64 instructions).
template <int P, int MODE, typename R>
__device__ __forceinline__ void make_pair(const FieldRef& s, const FieldRef& eta, const LatDesc& L, long long nitems,
                                          long long j, R xi[24], R phi[24]) {
  if (MODE == MODE_STANDARD || MODE == MODE_HPE) {
    load_r<P, R>(eta, L, nitems, j, xi);
    load_r<P, R>(s, L, nitems, j, phi);
  } else if (MODE == MODE_ONE_END) {
    load_r<P, R>(s, L, nitems, j, phi);
#pragma unroll
    for (int m = 0; m < 24; ++m) xi[m] = (m < 12) ? phi[m] : -phi[m];
  } else {  // generalised: xi = g5 s, phi = g5 eta - 2 i kappa amu s
    R e[24];
    load_r<P, R>(s, L, nitems, j, xi);
    load_r<P, R>(eta, L, nitems, j, e);
    const R k2 = (R)(2.0 * L.kappa * L.amu);
#pragma unroll
    for (int m = 0; m < 12; ++m) {
      const R sr = xi[2 * m], si = xi[2 * m + 1];
      if (m < 6) {
        phi[2 * m] = e[2 * m] + k2 * si;
        phi[2 * m + 1] = e[2 * m + 1] - k2 * sr;
      } else {
        phi[2 * m] = -e[2 * m] + k2 * si;
        phi[2 * m + 1] = -e[2 * m + 1] - k2 * sr;
        xi[2 * m] = -sr;
        xi[2 * m + 1] = -si;
      }
    }
  }
}

template <int P, int MODE, bool DERIV>
__global__ void contract_sites_kernel(Batch B, FieldRef s_e, FieldRef s_o, FieldRef eta_e, FieldRef eta_o,
                                      const double2* __restrict__ g64, double2* __restrict__ W) {
  const LatDesc& L = B.lat[0];
  const int npad = 1 << L.lognpad;
  const long long V = 2LL * L.Vh;
  const long long nfull = V * npad;
  const long long nitems = (long long)L.Vh * npad;
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nfull) return;
  const int col = (int)(j & (npad - 1));
  const int lex = (int)(j >> L.lognpad);
  const int ncomp = DERIV ? 80 : 16;
  if (col >= L.ncol) {
    for (int c = 0; c < ncomp; ++c) W[(size_t)c * nfull + j] = make_double2(0.0, 0.0);
    return;
  }
  int x = lex % L.X, r = lex / L.X;
  int y = r % L.Y;
  r /= L.Y;
  int z = r % L.Z, t = r / L.Z;
  const int p = (x + y + z + t) & 1;
  const long long jj = ((long long)(lex >> 1) << L.lognpad) + col;
  double xi[24], phi[24];
  make_pair<P, MODE, double>(p ? s_o : s_e, p ? eta_o : eta_e, L, nitems, jj, xi, phi);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      double re = 0.0, im = 0.0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double xr = xi[2 * (3 * a + c)], xim = xi[2 * (3 * a + c) + 1];
        double pr = phi[2 * (3 * b + c)], pim = phi[2 * (3 * b + c) + 1];
        re += xr * pr + xim * pim;
        im += xr * pim - xim * pr;
      }
      W[(size_t)(4 * a + b) * nfull + j] = make_double2(re, im);
    }
  if (DERIV) {
    for (int mu = 0; mu < 4; ++mu) {
      int xn = x, yn = y, zn = z, tn = t;
      double bc = 1.0;
      if (mu == 0) xn = (x + 1 == L.X) ? 0 : x + 1;
      if (mu == 1) yn = (y + 1 == L.Y) ? 0 : y + 1;
      if (mu == 2) zn = (z + 1 == L.Z) ? 0 : z + 1;
      if (mu == 3) {
        tn = (t + 1 == L.T) ? 0 : t + 1;
        if (t + 1 == L.T) bc = L.tbc;
      }
      const int lexn = lex_of(L, xn, yn, zn, tn);
      const long long jn = ((long long)(lexn >> 1) << L.lognpad) + col;
      double xif[24], phif[24];
      make_pair<P, MODE, double>(p ? s_e : s_o, p ? eta_e : eta_o, L, nitems, jn, xif, phif);
#pragma unroll
      for (int m = 0; m < 24; ++m) {
        xif[m] *= bc;
        phif[m] *= bc;
      }
      // U_mu(x), parity p, checkerboard index lex >> 1
      double u[18];
      const double2* gl = (const double2*)gauge_seg<G64R18>(g64, L) + (size_t)((p * 4 + mu) * 9) * L.Vh + (lex >> 1);
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        double2 c = gl[(size_t)k * L.Vh];
        u[2 * k] = c.x;
        u[2 * k + 1] = c.y;
      }
      double up[24], udp[24];  // U phi(x+mu), U^+ phi(x)
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          double r1 = 0, i1 = 0, r2 = 0, i2 = 0;
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            double ur = u[2 * (3 * a + b)], ui = u[2 * (3 * a + b) + 1];
            double vr = phif[2 * (3 * s + b)], vi = phif[2 * (3 * s + b) + 1];
            r1 += ur * vr - ui * vi;
            i1 += ur * vi + ui * vr;
            double wr = u[2 * (3 * b + a)], wi = -u[2 * (3 * b + a) + 1];
            double qr = phi[2 * (3 * s + b)], qi = phi[2 * (3 * s + b) + 1];
            r2 += wr * qr - wi * qi;
            i2 += wr * qi + wi * qr;
          }
          up[2 * (3 * s + a)] = r1;
          up[2 * (3 * s + a) + 1] = i1;
          udp[2 * (3 * s + a)] = r2;
          udp[2 * (3 * s + a) + 1] = i2;
        }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          double re = 0.0, im = 0.0;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            double xr = xi[2 * (3 * a + c)], xim = xi[2 * (3 * a + c) + 1];
            double pr = up[2 * (3 * b + c)], pim = up[2 * (3 * b + c) + 1];
            re += xr * pr + xim * pim;
            im += xr * pim - xim * pr;
            double fr = xif[2 * (3 * a + c)], fim = xif[2 * (3 * a + c) + 1];
            double qr = udp[2 * (3 * b + c)], qim = udp[2 * (3 * b + c) + 1];
            re -= fr * qr + fim * qim;
            im -= fr * qim - fim * qr;
          }
          W[(size_t)(16 * (mu + 1) + 4 * a + b) * nfull + j] = make_double2(re, im);
        }
    }
  }
}


// Fused per-site bilinears and x-direction DFT.  One CTA per (t, z, y) row;
// thread (x, column) forms the 16 (per derivative slot) components of its site
// in R, stores them to shared memory, and the CTA then writes
//   G1[comp][t][z][y][nx][col] = sum_x exp(-2 pi i nx x / X) C_comp(x, col)
// as R pairs.  Derivative slots d = 1..4 (mu = d - 1) are processed one at a
// time; their links come from the gauge copy G of the same precision as R
// (FP64 recon-18 for R = double, the FP32 copy otherwise), so the FP32 pipeline
// issues no FP64 instructions.
template <typename R>
struct RPair {
  R x, y;
};

#define DL_NXMAX 17  // x momenta per row: 2 floor(sqrt(P)) + 1 for |n|^2 <= P <= 64

// Phase table of the x DFT: pht[kx][x] = exp(-2 pi i (kx - mx) x / X) in R.
template <typename R>
__global__ void phase_table_kernel(int X, int mx, RPair<R>* pht) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int NX = 2 * mx + 1;
  if (e >= NX * X) return;
  const int kx = e / X, xx = e % X;
  int q = ((kx - mx) * xx) % X;
  if (q < 0) q += X;
  double sn, cn;
  sincospi(2.0 * (double)q / (double)X, &sn, &cn);
  pht[e].x = (R)cn;
  pht[e].y = (R)(-sn);
}

// MXT >= 0: the x-momentum extent mx is the compile-time MXT (no predicated
// iterations in the register-blocked DFT); MXT = -1: any mx <= 8.
// FP32 kernels with a compile-time x extent (the LP pipeline's) are compiled for three
// resident 256-thread CTAs per SM (80 registers), the others for the default.
template <int P, int MODE, bool DERIV, typename R, int G, int MXT>
__global__ void __launch_bounds__(256, (std::is_same<R, float>::value && MXT >= 0) ? 3 : 1) contract_x_kernel(Batch B, FieldRef s_e, FieldRef s_o, FieldRef eta_e,
                                                           FieldRef eta_o, const void* __restrict__ gbase, int mx,
                                                           int cwlog, const RPair<R>* __restrict__ phx,
                                                           RPair<R>* __restrict__ G1, Slices S) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const LatDesc& L = B.lat[0];
  const int lg = L.lognpad, npad = 1 << lg;
  const int cw = 1 << cwlog;                     // columns handled by this CTA
  const int mxk = MXT >= 0 ? MXT : mx;           // a constant for the compile-time extents
  const int NX = 2 * mxk + 1;
  typedef RPair<R> cr;
  cr* cs = (cr*)smem_raw;                        // [16][X][cw] site components
  cr* pht = cs + 16 * L.X * cw;                  // [NX][X] phases
  cr* part = pht + NX * L.X;                     // [4 or 2 parts][16][NX][cw] partial DFT sums
  const int row = blockIdx.x;                    // (k * Z + z) * Y + y for slice t = t0 + k dt
  const int y = row % L.Y, z = (row / L.Y) % L.Z, t = S.t0 + S.dt * (row / (L.Y * L.Z));
  const int x = threadIdx.x >> cwlog, cl = threadIdx.x & (cw - 1);
  const int col = blockIdx.y * cw + cl;
  for (int e = threadIdx.x; e < NX * L.X; e += blockDim.x) pht[e] = phx[e];
  const long long nitems = (long long)L.Vh << lg;
  const int lex = lex_of(L, x, y, z, t);
  const int p = (x + y + z + t) & 1;
  const bool live = col < L.ncol;
  R xi[24], phi[24];
  if (live) make_pair<P, MODE, R>(p ? s_o : s_e, p ? eta_o : eta_e, L, nitems, ((long long)(lex >> 1) << lg) + col, xi, phi);
  const long long nrows = (long long)S.ns * L.Z * L.Y;
  const int nd = DERIV ? 5 : 1;
  for (int d = 0; d < nd; ++d) {
    R cre[16], cim[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) cre[k] = cim[k] = 0;
    if (live) {
      if (d == 0) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            R re = 0, im = 0;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const R xr = xi[2 * (3 * a + c)], xim = xi[2 * (3 * a + c) + 1];
              const R pr = phi[2 * (3 * b + c)], pim = phi[2 * (3 * b + c) + 1];
              re += xr * pr + xim * pim;
              im += xr * pim - xim * pr;
            }
            cre[4 * a + b] = re;
            cim[4 * a + b] = im;
          }
      } else {
        const int mu = d - 1;
        int xn = x, yn = y, zn = z, tn = t;
        R bc = 1;
        if (mu == 0) xn = (x + 1 == L.X) ? 0 : x + 1;
        if (mu == 1) yn = (y + 1 == L.Y) ? 0 : y + 1;
        if (mu == 2) zn = (z + 1 == L.Z) ? 0 : z + 1;
        if (mu == 3) {
          tn = (t + 1 == L.T) ? 0 : t + 1;
          if (t + 1 == L.T) bc = (R)L.tbc;
        }
        const int lexn = lex_of(L, xn, yn, zn, tn);
        R xif[24], phif[24];
        make_pair<P, MODE, R>(p ? s_e : s_o, p ? eta_e : eta_o, L, nitems, ((long long)(lexn >> 1) << lg) + col, xif, phif);
        R u[18];
        GIO<G>::load(gauge_seg<G>(gbase, L), L.Vh, p, mu, lex >> 1, u);
        R up[24], udp[24];
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            R r1 = 0, i1 = 0, r2 = 0, i2 = 0;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
              const R ur = u[2 * (3 * a + b)], ui = u[2 * (3 * a + b) + 1];
              const R vr = phif[2 * (3 * sp + b)] * bc, vi = phif[2 * (3 * sp + b) + 1] * bc;
              r1 += ur * vr - ui * vi;
              i1 += ur * vi + ui * vr;
              const R wr = u[2 * (3 * b + a)], wi = -u[2 * (3 * b + a) + 1];
              const R qr = phi[2 * (3 * sp + b)], qi = phi[2 * (3 * sp + b) + 1];
              r2 += wr * qr - wi * qi;
              i2 += wr * qi + wi * qr;
            }
            up[2 * (3 * sp + a)] = r1;
            up[2 * (3 * sp + a) + 1] = i1;
            udp[2 * (3 * sp + a)] = r2;
            udp[2 * (3 * sp + a) + 1] = i2;
          }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            R re = 0, im = 0;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const R xr = xi[2 * (3 * a + c)], xim = xi[2 * (3 * a + c) + 1];
              const R pr = up[2 * (3 * b + c)], pim = up[2 * (3 * b + c) + 1];
              re += xr * pr + xim * pim;
              im += xr * pim - xim * pr;
              const R fr = xif[2 * (3 * a + c)] * bc, fim = xif[2 * (3 * a + c) + 1] * bc;
              const R qr = udp[2 * (3 * b + c)], qim = udp[2 * (3 * b + c) + 1];
              re -= fr * qr + fim * qim;
              im -= fr * qim - fim * qr;
            }
            cre[4 * a + b] = re;
            cim[4 * a + b] = im;
          }
      }
    }
    __syncthreads();  // previous slot's DFT has finished reading cs
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      cs[(k * L.X + x) * cw + cl].x = cre[k];
      cs[(k * L.X + x) * cw + cl].y = cim[k];
    }
    __syncthreads();
    // x DFT, register-blocked and paired in +-p_x.  The phases of the momenta +m and -m
    // are c -+ i s with the same c = cos(2 pi m x / X) and s = sin(2 pi m x / X), so with
    // Pc = sum_x v c and Q = sum_x v (-s)
    //   out(+m) = (Pc.re - Q.im, Pc.im + Q.re),   out(-m) = (Pc.re + Q.im, Pc.im - Q.re):
    // four multiply-adds per site for both momenta (eight for two plain DFT terms).  A task
    // (part of the row, component k, column or column pair) reads each site value once;
    // the parts are added in a fixed order.  FP32 runs two columns per task in packed
    // FP32x2 arithmetic over four parts of the row, the other types one column over two.
    constexpr int MC = MXT >= 0 ? MXT : (DL_NXMAX - 1) / 2;
    int nq = 2;
    bool packed = false;
    if constexpr (std::is_same<R, float>::value) packed = cw >= 2;
    if constexpr (std::is_same<R, float>::value) {
      if (packed) {
        nq = 4;
        const int hp = cw >> 1, qlen = (L.X + 3) >> 2;
        for (int task = threadIdx.x; task < 64 * hp; task += blockDim.x) {
          const int cp = task & (hp - 1), k = (task >> (cwlog - 1)) & 15, q = task >> (cwlog + 3);
          const int x0 = q * qlen, x1 = (x0 + qlen < L.X) ? x0 + qlen : L.X;
          float2 p0r = make_float2(0.f, 0.f), p0i = p0r, pcr[MC + 1], pci[MC + 1], qr[MC + 1], qi[MC + 1];
#pragma unroll
          for (int m = 0; m <= MC; ++m) pcr[m] = pci[m] = qr[m] = qi[m] = p0r;
          for (int xx = x0; xx < x1; ++xx) {
            const float4 v = *(const float4*)&cs[(k * L.X + xx) * cw + 2 * cp];
            const float2 vr = make_float2(v.x, v.z), vi = make_float2(v.y, v.w);
            p0r = add2(p0r, vr);
            p0i = add2(p0i, vi);
#pragma unroll
            for (int m = 1; m <= MC; ++m)
              if (MXT >= 0 || m <= mxk) {
                const cr w = pht[(mxk + m) * L.X + xx];
                const float2 c2 = dup2(w.x), s2 = dup2(w.y);
                pcr[m] = fma2(vr, c2, pcr[m]);
                pci[m] = fma2(vi, c2, pci[m]);
                qr[m] = fma2(vr, s2, qr[m]);
                qi[m] = fma2(vi, s2, qi[m]);
              }
          }
          cr* dst = part + (size_t)(q * 16 + k) * NX * cw + 2 * cp;
          dst[mxk * cw] = cr{p0r.x, p0i.x};
          dst[mxk * cw + 1] = cr{p0r.y, p0i.y};
#pragma unroll
          for (int m = 1; m <= MC; ++m)
            if (MXT >= 0 || m <= mxk) {
              dst[(mxk + m) * cw] = cr{pcr[m].x - qi[m].x, pci[m].x + qr[m].x};
              dst[(mxk + m) * cw + 1] = cr{pcr[m].y - qi[m].y, pci[m].y + qr[m].y};
              dst[(mxk - m) * cw] = cr{pcr[m].x + qi[m].x, pci[m].x - qr[m].x};
              dst[(mxk - m) * cw + 1] = cr{pcr[m].y + qi[m].y, pci[m].y - qr[m].y};
            }
        }
      }
    }
    if (!packed) {
      const int qlen = (L.X + 1) >> 1;
      for (int task = threadIdx.x; task < 32 * cw; task += blockDim.x) {
        const int cc = task & (cw - 1);
        const int k = (task >> cwlog) & 15;
        const int q = task >> (cwlog + 4);
        const int x0 = q * qlen, x1 = (x0 + qlen < L.X) ? x0 + qlen : L.X;
        R p0r = 0, p0i = 0, pcr[MC + 1], pci[MC + 1], qr[MC + 1], qi[MC + 1];
#pragma unroll
        for (int m = 0; m <= MC; ++m) pcr[m] = pci[m] = qr[m] = qi[m] = 0;
        for (int xx = x0; xx < x1; ++xx) {
          const cr v = cs[(k * L.X + xx) * cw + cc];
          p0r += v.x;
          p0i += v.y;
#pragma unroll
          for (int m = 1; m <= MC; ++m)
            if (MXT >= 0 || m <= mxk) {
              const cr w = pht[(mxk + m) * L.X + xx];
              pcr[m] += v.x * w.x;
              pci[m] += v.y * w.x;
              qr[m] += v.x * w.y;
              qi[m] += v.y * w.y;
            }
        }
        cr* dst = part + (size_t)(q * 16 + k) * NX * cw + cc;
        dst[mxk * cw] = cr{p0r, p0i};
#pragma unroll
        for (int m = 1; m <= MC; ++m)
          if (MXT >= 0 || m <= mxk) {
            dst[(mxk + m) * cw] = cr{pcr[m] - qi[m], pci[m] + qr[m]};
            dst[(mxk - m) * cw] = cr{pcr[m] + qi[m], pci[m] - qr[m]};
          }
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 16 * NX * cw; e += blockDim.x) {
      const int cc = e & (cw - 1);
      const int kx = (e >> cwlog) % NX;
      const int k = (e >> cwlog) / NX;
      cr a = part[(k * NX + kx) * cw + cc];
      for (int q = 1; q < nq; ++q) {
        const cr b = part[((q * 16 + k) * NX + kx) * cw + cc];
        a.x += b.x;
        a.y += b.y;
      }
      G1[(((long long)(16 * d + k) * nrows + row) * NX + kx) * npad + blockIdx.y * cw + cc] = a;
    }
  }
}

__global__ void phase_kernel(int len, double2* ph) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= len) return;
  double s, c;
  sincospi(2.0 * (double)q / (double)len, &s, &c);
  ph[q] = make_double2(c, -s);  // exp(-2 pi i q / len)
}

// out[b][k][s] = sum_j in[b][j][s] exp(-2 pi i (k - m) j / len), accumulated in R.
// One CTA per (b, tile of DL_DFT_TILE s): the [len x tile] input slab is staged
// in shared memory with coalesced loads, then the CTA's threads compute the
// (2m+1) x tile outputs from shared memory.
#define DL_DFT_TILE 64
template <typename R>
__global__ void __launch_bounds__(256) dft_kernel(const RPair<R>* __restrict__ in, RPair<R>* __restrict__ out, long long nb,
                                                  int len, long long stride, int m, const double2* __restrict__ ph) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  typedef RPair<R> cr;
  cr* slab = (cr*)smem_raw;            // [len][DL_DFT_TILE]
  cr* phs = slab + len * DL_DFT_TILE;  // [len]
  const long long ntile = (stride + DL_DFT_TILE - 1) / DL_DFT_TILE;
  const long long b = blockIdx.x / ntile;
  const long long s0 = (blockIdx.x % ntile) * DL_DFT_TILE;
  const int tw = (int)((stride - s0) < DL_DFT_TILE ? (stride - s0) : DL_DFT_TILE);
  for (int q = threadIdx.x; q < len; q += blockDim.x) {
    phs[q].x = (R)ph[q].x;
    phs[q].y = (R)ph[q].y;
  }
  const cr* src = in + b * len * stride + s0;
  for (int e = threadIdx.x; e < len * DL_DFT_TILE; e += blockDim.x) {
    const int j = e / DL_DFT_TILE, ss = e % DL_DFT_TILE;
    if (ss < tw) slab[e] = src[(long long)j * stride + ss];
  }
  __syncthreads();
  // the momenta +mm and -mm share c and s of their phases c -+ i s: with Pc = sum v c and
  // Q = sum v (-s), out(+mm) = (Pc.re - Q.im, Pc.im + Q.re), out(-mm) = (Pc.re + Q.im, Pc.im - Q.re)
  const int nk = 2 * m + 1;
  for (int o = threadIdx.x; o < (m + 1) * DL_DFT_TILE; o += blockDim.x) {
    const int mm = o / DL_DFT_TILE, ss = o % DL_DFT_TILE;
    if (ss >= tw) continue;
    const int n = mm % len;
    R pr = 0, pi = 0, qr = 0, qi = 0;
    if (mm == 0) {
#pragma unroll 4
      for (int jx = 0; jx < len; ++jx) {
        const cr v = slab[jx * DL_DFT_TILE + ss];
        pr += v.x;
        pi += v.y;
      }
      out[(b * nk + m) * stride + s0 + ss] = cr{pr, pi};
      continue;
    }
    int q = 0;
#pragma unroll 4
    for (int jx = 0; jx < len; ++jx) {
      const cr v = slab[jx * DL_DFT_TILE + ss];
      const cr w = phs[q];
      pr += v.x * w.x;
      pi += v.y * w.x;
      qr += v.x * w.y;
      qi += v.y * w.y;
      q += n;
      if (q >= len) q -= len;
    }
    out[(b * nk + m + mm) * stride + s0 + ss] = cr{pr - qi, pi + qr};
    out[(b * nk + m - mm) * stride + s0 + ss] = cr{pr + qi, pi - qr};
  }
}

// out[col][t][ip][d][ab] (+)= pre * finalised G3 (G3 holds R pairs)
template <typename R>
__global__ void finalize_kernel(LatDesc L, int npad, int nd, int np, const int* __restrict__ mom, int mx, int my, int mz,
                                const RPair<R>* __restrict__ G3,
                                double pre_re, double pre_im, double2* out, int accumulate, Slices S) {
  const long long tot = (long long)L.ncol * L.T * np * nd * 16;
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= tot) return;
  int ab = (int)(idx % 16);
  long long r = idx / 16;
  int d = (int)(r % nd);
  r /= nd;
  int ip = (int)(r % np);
  r /= np;
  int t = (int)(r % L.T);
  int col = (int)(r / L.T);
  int nx = mom[3 * ip], ny = mom[3 * ip + 1], nz = mom[3 * ip + 2];
  const int NX = 2 * mx + 1, NY = 2 * my + 1, NZ = 2 * mz + 1;
  const long long cube = (long long)NZ * NY * NX * npad;
  // G3 holds the covered slices only (index k of t = t0 + k dt); other slices are zero
  auto g = [&](int comp, int tt) -> double2 {
    const int k = slice_index(S, tt);
    if (k < 0) return make_double2(0.0, 0.0);
    long long o = ((long long)comp * S.ns + k) * cube + (((long long)(nz + mz) * NY + (ny + my)) * NX + (nx + mx)) * npad + col;
    return make_double2((double)G3[o].x, (double)G3[o].y);
  };
  double2 v;
  if (d == 0) {
    v = g(ab, t);
  } else if (d < 4) {
    double2 h = g(16 * d + ab, t);
    int nmu = (d == 1) ? nx : (d == 2 ? ny : nz);
    int lmu = (d == 1) ? L.X : (d == 2 ? L.Y : L.Z);
    double s, c;
    sincospi(2.0 * (double)nmu / (double)lmu, &s, &c);
    double fr = 0.25 * (1.0 + c), fi = -0.25 * s;  // (1 + exp(-i p_mu)) / 4
    v = make_double2(fr * h.x - fi * h.y, fr * h.y + fi * h.x);
  } else {
    double2 h0 = g(64 + ab, t), h1 = g(64 + ab, (t == 0) ? L.T - 1 : t - 1);
    v = make_double2(0.25 * (h0.x + h1.x), 0.25 * (h0.y + h1.y));
  }
  double2 res = make_double2(pre_re * v.x - pre_im * v.y, pre_re * v.y + pre_im * v.x);
  if (accumulate) {
    double2 o = out[idx];
    res.x += o.x;
    res.y += o.y;
  }
  out[idx] = res;
}

// Exact hopping-parameter-expansion terms for local insertions at one site:
// E = B + kappa^2 B S B with S = sum_mu [(1 - g_mu) B (1 + g_mu) + (1 + g_mu) B (1 - g_mu)],
// colour trace 3; written in the bilinear convention C_ab = 3 E_ba.
struct c4 {
  double r[4][4], i[4][4];
};
__device__ void mm4(const c4& a, const c4& b, c4& o) {
  for (int x = 0; x < 4; ++x)
    for (int y = 0; y < 4; ++y) {
      double re = 0, im = 0;
      for (int k = 0; k < 4; ++k) {
        re += a.r[x][k] * b.r[k][y] - a.i[x][k] * b.i[k][y];
        im += a.r[x][k] * b.i[k][y] + a.i[x][k] * b.r[k][y];
      }
      o.r[x][y] = re;
      o.i[x][y] = im;
    }
}
__global__ void hpe_exact_kernel(double kappa, double amu, int flavour, double2* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  // chiral gammas: g_k = [[0, -i s_k], [i s_k, 0]], g_t = [[0, 1], [1, 0]]
  c4 g[4];
  for (int mu = 0; mu < 4; ++mu)
    for (int x = 0; x < 4; ++x)
      for (int y = 0; y < 4; ++y) g[mu].r[x][y] = g[mu].i[x][y] = 0.0;
  // sigma_1 = [[0,1],[1,0]], sigma_2 = [[0,-i],[i,0]], sigma_3 = diag(1,-1)
  // -i s_1 = [[0,-i],[-i,0]]
  g[0].i[0][3] = -1; g[0].i[1][2] = -1; g[0].i[2][1] = 1; g[0].i[3][0] = 1;
  // -i s_2 = [[0,-1],[1,0]], i s_2 = [[0,1],[-1,0]]
  g[1].r[0][3] = -1; g[1].r[1][2] = 1; g[1].r[2][1] = 1; g[1].r[3][0] = -1;
  // -i s_3 = diag(-i, i), i s_3 = diag(i, -i)
  g[2].i[0][2] = -1; g[2].i[1][3] = 1; g[2].i[2][0] = 1; g[2].i[3][1] = -1;
  g[3].r[0][2] = 1; g[3].r[1][3] = 1; g[3].r[2][0] = 1; g[3].r[3][1] = 1;
  // B = (1 + i w g5)^-1 = (1 - i w g5) / (1 + w^2), w = 2 kappa amu f
  const double w = 2.0 * kappa * amu * flavour, n = 1.0 / (1.0 + w * w);
  c4 Bm, S, T1, T2, P1, P2;
  for (int x = 0; x < 4; ++x)
    for (int y = 0; y < 4; ++y) {
      Bm.r[x][y] = (x == y) ? n : 0.0;
      Bm.i[x][y] = (x == y) ? -w * n * (x < 2 ? 1.0 : -1.0) : 0.0;
      S.r[x][y] = S.i[x][y] = 0.0;
    }
  for (int mu = 0; mu < 4; ++mu)
    for (int sg = -1; sg <= 1; sg += 2) {
      for (int x = 0; x < 4; ++x)
        for (int y = 0; y < 4; ++y) {
          double id = (x == y) ? 1.0 : 0.0;
          P1.r[x][y] = id - sg * g[mu].r[x][y];
          P1.i[x][y] = -sg * g[mu].i[x][y];
          P2.r[x][y] = id + sg * g[mu].r[x][y];
          P2.i[x][y] = sg * g[mu].i[x][y];
        }
      mm4(P1, Bm, T1);
      mm4(T1, P2, T2);
      for (int x = 0; x < 4; ++x)
        for (int y = 0; y < 4; ++y) {
          S.r[x][y] += T2.r[x][y];
          S.i[x][y] += T2.i[x][y];
        }
    }
  mm4(Bm, S, T1);
  mm4(T1, Bm, T2);
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      double er = Bm.r[b][a] + kappa * kappa * T2.r[b][a];
      double ei = Bm.i[b][a] + kappa * kappa * T2.i[b][a];
      out[4 * a + b] = make_double2(3.0 * er, 3.0 * ei);
    }
}

__global__ void add_exact_kernel(LatDesc L, int np, int nd, int ip0, const double2* __restrict__ ex, double scale,
                                 double2* out, Slices S) {
  long long tot = (long long)L.ncol * L.T * 16;
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= tot) return;
  int ab = (int)(idx % 16);
  long long r = idx / 16;
  int t = (int)(r % L.T);
  int col = (int)(r / L.T);
  if (slice_index(S, t) < 0) return;  // the source is zero on this slice: no exact part either
  long long o = ((((long long)col * L.T + t) * np + ip0) * nd + 0) * 16 + ab;
  out[o].x += scale * ex[ab].x;
  out[o].y += scale * ex[ab].y;
}


// acc[k] += sign * sum_col (blk[col][k] - sub[col][k])  (sub may be null)
__global__ void col_accumulate_kernel(const double2* __restrict__ blk, const double2* __restrict__ sub, int ncol,
                                      long long per_col, double sign, double2* acc) {
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= per_col) return;
  double re = 0.0, im = 0.0;
  for (int col = 0; col < ncol; ++col) {
    double2 v = blk[(long long)col * per_col + k];
    re += v.x;
    im += v.y;
    if (sub) {
      double2 w = sub[(long long)col * per_col + k];
      re -= w.x;
      im -= w.y;
    }
  }
  acc[k].x += sign * re;
  acc[k].y += sign * im;
}

// Per-column scalar observables at zero momentum summed over t:
//   sigma = sum_ab (i g5)_ab L1_ab,   axial = sum_ab (g_z g5)_ab L2_ab
// with g_z g5 = [[0, i s3], [i s3, 0]] in the chiral basis.
__global__ void observables_kernel(const double2* __restrict__ l1, const double2* __restrict__ l2, int ncol, int T, int np,
                                   int nd, int ip0, double* obs) {
  int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= ncol) return;
  double sr = 0, si = 0, ar = 0, ai = 0;
  for (int t = 0; t < T; ++t) {
    long long o = ((((long long)col * T + t) * np + ip0) * nd) * 16;
    const double2* a = l1 + o;
    const double2* b = l2 + o;
    // i g5 = diag(i, i, -i, -i): i * (C00 + C11 - C22 - C33)
    double dr = a[0].x + a[5].x - a[10].x - a[15].x, di = a[0].y + a[5].y - a[10].y - a[15].y;
    sr += -di;
    si += dr;
    // (0,2) = i, (1,3) = -i, (2,0) = i, (3,1) = -i
    double er = b[2].x - b[7].x + b[8].x - b[13].x, ei = b[2].y - b[7].y + b[8].y - b[13].y;
    ar += -ei;
    ai += er;
  }
  obs[4 * col + 0] = sr;
  obs[4 * col + 1] = si;
  obs[4 * col + 2] = ar;
  obs[4 * col + 3] = ai;
}

// out = a * x + b * y
__global__ void combine_kernel(const double2* x, const double2* y, double a, double b, long long n, double2* out) {
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  out[k] = make_double2(a * x[k].x + b * y[k].x, a * x[k].y + b * y[k].y);
}

}  // namespace

namespace dl {

cudaError_t col_accumulate(const double2* blk, const double2* sub, int ncol, long long per_col, double sign, double2* acc,
                           cudaStream_t st) {
  if (per_col <= 0) return cudaSuccess;
  DL_COUNT();
  col_accumulate_kernel<<<(int)((per_col + 255) / 256), 256, 0, st>>>(blk, sub, ncol, per_col, sign, acc);
  return cudaGetLastError();
}

cudaError_t observables(const double2* l1, const double2* l2, int ncol, int T, int np, int nd, int ip0, double* obs,
                        cudaStream_t st) {
  DL_COUNT();
  observables_kernel<<<(ncol + 31) / 32, 32, 0, st>>>(l1, l2, ncol, T, np, nd, ip0, obs);
  return cudaGetLastError();
}

cudaError_t combine(const double2* x, const double2* y, double a, double b, long long n, double2* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  DL_COUNT();
  combine_kernel<<<(int)((n + 255) / 256), 256, 0, st>>>(x, y, a, b, n, out);
  return cudaGetLastError();
}

cudaError_t contract_sites(const Batch& B, int prec, int mode, int with_deriv, FieldRef s_e, FieldRef s_o, FieldRef eta_e,
                           FieldRef eta_o, const void* g64, double2* W, cudaStream_t st) {
  const LatDesc& L = B.lat[0];
  long long nfull = (2LL * L.Vh) << L.lognpad;
  int g = (int)((nfull + 127) / 128);
  const double2* gg = (const double2*)g64;
#define CS(PR, MD)                                                                                          \
  if (prec == PR && mode == MD) {                                                                           \
    DL_COUNT();                                                                                             \
    if (with_deriv) contract_sites_kernel<PR, MD, true><<<g, 128, 0, st>>>(B, s_e, s_o, eta_e, eta_o, gg, W);  \
    else contract_sites_kernel<PR, MD, false><<<g, 128, 0, st>>>(B, s_e, s_o, eta_e, eta_o, gg, W);          \
    return cudaGetLastError();                                                                              \
  }
  CS(P64, 0) CS(P64, 1) CS(P64, 2) CS(P64, 3) CS(P32, 0) CS(P32, 1) CS(P32, 2) CS(P32, 3)
  CS(PDF, 0) CS(PDF, 1) CS(PDF, 2) CS(PDF, 3)
#undef CS
  return cudaErrorInvalidValue;
}

template <int PR, int MD, bool DV, typename R, int G, int MXT>
cudaError_t launch_cx(const Batch& B, dim3 grid, int threads, int cwlog, int mx, FieldRef s_e, FieldRef s_o,
                      FieldRef eta_e, FieldRef eta_o, const void* gb, double2* phx, double2* G1, Slices S,
                      cudaStream_t st) {
  const LatDesc& L = B.lat[0];
  const int NX = 2 * mx + 1;
  // site components, phase table, partial x-DFT sums (four row parts for FP32, two otherwise)
  const int nq = std::is_same<R, float>::value ? 4 : 2;
  const size_t smem = (size_t)(16 * L.X * (1 << cwlog) + NX * L.X + 16 * nq * NX * (1 << cwlog)) * 2 * sizeof(R);
  if (smem > 200000) return cudaErrorInvalidValue;
  DL_COUNT();
  phase_table_kernel<R><<<(NX * L.X + 255) / 256, 256, 0, st>>>(L.X, mx, (RPair<R>*)phx);
  DL_CUDA_TRY(cudaFuncSetAttribute(contract_x_kernel<PR, MD, DV, R, G, MXT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200000));
  DL_COUNT();
  contract_x_kernel<PR, MD, DV, R, G, MXT><<<grid, threads, smem, st>>>(B, s_e, s_o, eta_e, eta_o, gb, mx, cwlog,
                                                                         (const RPair<R>*)phx, (RPair<R>*)G1, S);
  return cudaGetLastError();
}

// One (precision, estimator, derivative) combination: its arithmetic type and gauge
// copy, and for the local contractions a kernel per x extent (FP32: mx <= 3; double-float:
// mx = 3, the extent of |n|^2 <= 9).
template <int PR, int MD, bool DV>
cudaError_t dispatch_cx(const Batch& B, dim3 grid, int threads, int cwlog, int mx, FieldRef s_e, FieldRef s_o,
                        FieldRef eta_e, FieldRef eta_o, const void* g64, const void* g32, int rec32, double2* phx,
                        double2* G1, Slices S, cudaStream_t st) {
#define ARGS B, grid, threads, cwlog, mx, s_e, s_o, eta_e, eta_o
  if constexpr (PR == P64) {
    return launch_cx<PR, MD, DV, double, G64R18, -1>(ARGS, g64, phx, G1, S, st);
  } else if constexpr (PR == PDF) {
    if constexpr (!DV) {
      if (mx == 3) return launch_cx<PR, MD, DV, dfloat, GDF18, 3>(ARGS, g64, phx, G1, S, st);  // |n|^2 <= 9 .. 15
    }
    return launch_cx<PR, MD, DV, dfloat, GDF18, -1>(ARGS, g64, phx, G1, S, st);
  } else {
    if constexpr (!DV) {
      if (rec32 == 12) {
        switch (mx) {
          case 0: return launch_cx<PR, MD, DV, float, G32R12, 0>(ARGS, g32, phx, G1, S, st);
          case 1: return launch_cx<PR, MD, DV, float, G32R12, 1>(ARGS, g32, phx, G1, S, st);
          case 2: return launch_cx<PR, MD, DV, float, G32R12, 2>(ARGS, g32, phx, G1, S, st);
          case 3: return launch_cx<PR, MD, DV, float, G32R12, 3>(ARGS, g32, phx, G1, S, st);
          default: break;
        }
      } else {
        switch (mx) {
          case 0: return launch_cx<PR, MD, DV, float, G32R8, 0>(ARGS, g32, phx, G1, S, st);
          case 1: return launch_cx<PR, MD, DV, float, G32R8, 1>(ARGS, g32, phx, G1, S, st);
          case 2: return launch_cx<PR, MD, DV, float, G32R8, 2>(ARGS, g32, phx, G1, S, st);
          case 3: return launch_cx<PR, MD, DV, float, G32R8, 3>(ARGS, g32, phx, G1, S, st);
          default: break;
        }
      }
    }
    if (rec32 == 12) return launch_cx<PR, MD, DV, float, G32R12, -1>(ARGS, g32, phx, G1, S, st);
    return launch_cx<PR, MD, DV, float, G32R8, -1>(ARGS, g32, phx, G1, S, st);
  }
#undef ARGS
}

}  // namespace dl

namespace dl {

cudaError_t contract_x(const Batch& B, int prec, int mode, int with_deriv, FieldRef s_e, FieldRef s_o, FieldRef eta_e,
                       FieldRef eta_o, const void* g64, const void* g32, int rec32, int mx, double2* phx, double2* G1,
                       Slices S, cudaStream_t st) {
  const LatDesc& L = B.lat[0];
  const int npad = 1 << L.lognpad;
  int cwlog = L.lognpad;
  while (cwlog > 0 && (L.X << cwlog) > 256) --cwlog;  // X * cw <= 256 threads per CTA
  const int threads = L.X << cwlog;
  if (threads > 256 || threads < 1) return cudaErrorInvalidValue;
  if (prec == P32 && rec32 != 12 && rec32 != 8) return cudaErrorInvalidValue;
  if (2 * mx + 1 > DL_NXMAX) return cudaErrorInvalidValue;
  if (S.ns < 1 || S.dt < 1 || S.t0 < 0 || S.t0 + S.dt * (S.ns - 1) >= L.T) return cudaErrorInvalidValue;
  if (with_deriv && S.ns != L.T) return cudaErrorInvalidValue;  // the derivative reaches t - 1 and t + 1
  const dim3 grid(S.ns * L.Z * L.Y, npad >> cwlog);
#define CX(PR, MD)                                                                                                  \
  if (prec == PR && mode == MD)                                                                                    \
    return with_deriv ? dispatch_cx<PR, MD, true>(B, grid, threads, cwlog, mx, s_e, s_o, eta_e, eta_o, g64, g32,   \
                                                  rec32, phx, G1, S, st)                                           \
                      : dispatch_cx<PR, MD, false>(B, grid, threads, cwlog, mx, s_e, s_o, eta_e, eta_o, g64, g32,  \
                                                   rec32, phx, G1, S, st);
  CX(P64, 0) CX(P64, 1) CX(P64, 2) CX(P64, 3)
  CX(P32, 0) CX(P32, 1) CX(P32, 2) CX(P32, 3)
  CX(PDF, 0) CX(PDF, 1) CX(PDF, 2) CX(PDF, 3)
#undef CX
  return cudaErrorInvalidValue;
}

cudaError_t dft_pass(const double2* in, double2* out, long long nb, int len, long long stride, int m, double2* phase,
                     int fp32, cudaStream_t st) {
  DL_COUNT();
  phase_kernel<<<(len + 63) / 64, 64, 0, st>>>(len, phase);
  const long long ntile = (stride + DL_DFT_TILE - 1) / DL_DFT_TILE;
  const long long g = nb * ntile;
  if (g <= 0) return cudaSuccess;
  if (g > 0x7fffffffLL) return cudaErrorInvalidValue;
  DL_COUNT();
  if ((size_t)(len * DL_DFT_TILE + len) * 2 * (fp32 == 1 ? sizeof(float) : sizeof(double)) > 200000)
    return cudaErrorInvalidValue;  // extents up to ~190 (FP64) / ~380 (FP32) sites
  if (fp32 == 2) {  // double-float pairs
    const size_t smem = (size_t)(len * DL_DFT_TILE + len) * 2 * sizeof(dfloat);
    DL_CUDA_TRY(cudaFuncSetAttribute(dft_kernel<dfloat>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200000));
    dft_kernel<dfloat><<<(int)g, 256, smem, st>>>((const RPair<dfloat>*)in, (RPair<dfloat>*)out, nb, len, stride, m,
                                                 phase);
  } else if (fp32 == 1) {  // in and out hold float pairs
    const size_t smem = (size_t)(len * DL_DFT_TILE + len) * 2 * sizeof(float);
    DL_CUDA_TRY(cudaFuncSetAttribute(dft_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200000));
    dft_kernel<float><<<(int)g, 256, smem, st>>>((const RPair<float>*)in, (RPair<float>*)out, nb, len, stride, m, phase);
  } else {
    const size_t smem = (size_t)(len * DL_DFT_TILE + len) * 2 * sizeof(double);
    DL_CUDA_TRY(cudaFuncSetAttribute(dft_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200000));
    dft_kernel<double><<<(int)g, 256, smem, st>>>((const RPair<double>*)in, (RPair<double>*)out, nb, len, stride, m,
                                                 phase);
  }
  return cudaGetLastError();
}

cudaError_t contract_finalize(const Batch& B, int with_deriv, int np, const int* mom_dev, int mx, int my, int mz,
                              const double2* G3, int fp32, double pre_re, double pre_im, double2* out, int accumulate,
                              Slices S, cudaStream_t st) {
  const LatDesc& L = B.lat[0];
  int nd = with_deriv ? 5 : 1;
  long long tot = (long long)L.ncol * L.T * np * nd * 16;
  if (tot == 0) return cudaSuccess;
  DL_COUNT();
  if (fp32 == 2)
    finalize_kernel<dfloat><<<(int)((tot + 255) / 256), 256, 0, st>>>(L, 1 << L.lognpad, nd, np, mom_dev, mx, my, mz,
                                                                     (const RPair<dfloat>*)G3, pre_re, pre_im, out,
                                                                     accumulate, S);
  else if (fp32 == 1)
    finalize_kernel<float><<<(int)((tot + 255) / 256), 256, 0, st>>>(L, 1 << L.lognpad, nd, np, mom_dev, mx, my, mz,
                                                                    (const RPair<float>*)G3, pre_re, pre_im, out,
                                                                    accumulate, S);
  else
    finalize_kernel<double><<<(int)((tot + 255) / 256), 256, 0, st>>>(L, 1 << L.lognpad, nd, np, mom_dev, mx, my, mz,
                                                                     (const RPair<double>*)G3, pre_re, pre_im, out,
                                                                     accumulate, S);
  return cudaGetLastError();
}

cudaError_t hpe_exact(double kappa, double amu, int flavour, double2* out16, cudaStream_t st) {
  DL_COUNT();
  hpe_exact_kernel<<<1, 32, 0, st>>>(kappa, amu, flavour, out16);
  return cudaGetLastError();
}

cudaError_t add_exact_p0(const Batch& B, int np, int nd, int ip0, const double2* exact16, double scale, double2* out,
                         Slices S, cudaStream_t st) {
  const LatDesc& L = B.lat[0];
  long long tot = (long long)L.ncol * L.T * 16;
  DL_COUNT();
  add_exact_kernel<<<(int)((tot + 255) / 256), 256, 0, st>>>(L, np, nd, ip0, exact16, scale, out, S);
  return cudaGetLastError();
}

}  // namespace dl
