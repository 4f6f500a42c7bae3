// Kernels of the learned preconditioner: a gauge-covariant network of
// parallel-transport convolution layers (no counterpart in the paper).  A layer
// maps C_in channel fields to C_out:
//   y_o(x) = sum_i [ sum_b W[0][b][o][i] L_b x_i(x)
//                    + sum_mu sum_b W[1+2mu][b][o][i] H_b U_mu(x) x_i(x+mu)
//                    + sum_mu sum_b W[2+2mu][b][o][i] H_b U_mu(x-mu)^+ x_i(x-mu) ]
// with L_b in {1, g5} and H_b in {1, g_mu, g5, g5 g_mu}; weights are complex FP32
// [9][4][C_out][C_in].  Channels are the columns of the even-odd field layout, so
// the 16 channels of a site sit next to each other.  A CTA covers 16 sites of one
// parity; its links and neighbour indices are staged in shared memory.
#include "dl_internal.cuh"
#include "dl_kernels.h"

namespace {

constexpr int NS = 16;  // sites per CTA (forward, input gradient)

__device__ __forceinline__ float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) { return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }  // conj(a) b

// gamma_mu v in the chiral basis: (g v)_up = G v_dn, (g v)_dn = G^+ v_up with
// G_k = -i sigma_k (k = x, y, z), G_t = 1.  v, o: [spin][colour][re, im].
template <int MU>
__device__ __forceinline__ void gamma_apply(const float* v, float* o) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float u0r = v[2 * c], u0i = v[2 * c + 1], u1r = v[6 + 2 * c], u1i = v[7 + 2 * c];
    const float d2r = v[12 + 2 * c], d2i = v[13 + 2 * c], d3r = v[18 + 2 * c], d3i = v[19 + 2 * c];
    float a0r, a0i, a1r, a1i, b0r, b0i, b1r, b1i;
    if (MU == 0) {  // G d = (-i d3, -i d2), G^+ u = (i u1, i u0)
      a0r = d3i; a0i = -d3r; a1r = d2i; a1i = -d2r;
      b0r = -u1i; b0i = u1r; b1r = -u0i; b1i = u0r;
    } else if (MU == 1) {  // G d = (-d3, d2), G^+ u = (u1, -u0)
      a0r = -d3r; a0i = -d3i; a1r = d2r; a1i = d2i;
      b0r = u1r; b0i = u1i; b1r = -u0r; b1i = -u0i;
    } else if (MU == 2) {  // G d = (-i d2, i d3), G^+ u = (i u0, -i u1)
      a0r = d2i; a0i = -d2r; a1r = -d3i; a1i = d3r;
      b0r = -u0i; b0i = u0r; b1r = u1i; b1i = -u1r;
    } else {  // G = 1
      a0r = d2r; a0i = d2i; a1r = d3r; a1i = d3i;
      b0r = u0r; b0i = u0i; b1r = u1r; b1i = u1i;
    }
    o[2 * c] = a0r; o[2 * c + 1] = a0i; o[6 + 2 * c] = a1r; o[7 + 2 * c] = a1i;
    o[12 + 2 * c] = b0r; o[13 + 2 * c] = b0i; o[18 + 2 * c] = b1r; o[19 + 2 * c] = b1i;
  }
}

__device__ __forceinline__ void gamma_apply_rt(int mu, const float* v, float* o) {
  switch (mu) {
    case 0: gamma_apply<0>(v, o); break;
    case 1: gamma_apply<1>(v, o); break;
    case 2: gamma_apply<2>(v, o); break;
    default: gamma_apply<3>(v, o); break;
  }
}

// out = U v (dag = false) or U^+ v, colour matrix on all four spins
__device__ __forceinline__ void colour_mul(const float* u, const float* v, float* out, bool dag) {
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float re = 0.f, im = 0.f;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        float ur, ui;
        if (dag) { ur = u[2 * (3 * b + a)]; ui = -u[2 * (3 * b + a) + 1]; }
        else { ur = u[2 * (3 * a + b)]; ui = u[2 * (3 * a + b) + 1]; }
        const float vr = v[6 * s + 2 * b], vi = v[6 * s + 2 * b + 1];
        re += ur * vr - ui * vi;
        im += ur * vi + ui * vr;
      }
      out[6 * s + 2 * a] = re;
      out[6 * s + 2 * a + 1] = im;
    }
}

// Stage the 8 links (boundary factor folded in) and neighbour indices of NS
// consecutive sites of parity p starting at site0.
template <int G>
__device__ __forceinline__ void stage_links(const LatDesc& L, int p, int site0, int ns, const void* gb, float* su, int* snb) {
  for (int task = threadIdx.x; task < 8 * ns; task += blockDim.x) {
    const int sl = task % ns, d = task / ns;
    const int i = site0 + sl;
    if (i < L.Vh) {
      int x, y, z, t;
      cb_coords(L, i, p, x, y, z, t);
      const int mu = d >> 1;
      const bool bwd = d & 1;
      bool crosses = false;
      int xn = x, yn = y, zn = z, tn = t;
      if (mu == 0) xn = bwd ? (x == 0 ? L.X - 1 : x - 1) : (x + 1 == L.X ? 0 : x + 1);
      else if (mu == 1) yn = bwd ? (y == 0 ? L.Y - 1 : y - 1) : (y + 1 == L.Y ? 0 : y + 1);
      else if (mu == 2) zn = bwd ? (z == 0 ? L.Z - 1 : z - 1) : (z + 1 == L.Z ? 0 : z + 1);
      else {
        crosses = bwd ? (t == 0) : (t + 1 == L.T);
        tn = bwd ? (t == 0 ? L.T - 1 : t - 1) : (t + 1 == L.T ? 0 : t + 1);
      }
      const int nb = lex_of(L, xn, yn, zn, tn) >> 1;
      float u[18];
      GIO<G>::load(gb, L.Vh, bwd ? 1 - p : p, mu, bwd ? nb : i, u);
      const float f = crosses ? (float)L.tbc : 1.f;
      float* dst = su + (d * ns + sl) * 18;
#pragma unroll
      for (int e = 0; e < 18; ++e) dst[e] = u[e] * f;
      snb[d * ns + sl] = nb;
    }
  }
}

// ------------------------------------------------------------------ forward
template <int P, int G>
__global__ void __launch_bounds__(256) nn_fwd_kernel(LatDesc L, int p, FieldRef xe, FieldRef xo, FieldRef y,
                                                     const void* __restrict__ g32, const float2* __restrict__ W, int CI,
                                                     int CO, int lgin, int lgout) {
  __shared__ float su[8 * NS * 18];
  __shared__ int snb[8 * NS];
  __shared__ float Z[NS][9][24];
  __shared__ float Zg[NS][9][24];
  const int site0 = blockIdx.x * NS;
  stage_links<G>(L, p, site0, NS, gauge_seg<G>(g32, L), su, snb);
  __syncthreads();
  const int s = threadIdx.x >> 4, j = threadIdx.x & 15;
  const int site = site0 + s;
  const bool live = site < L.Vh;
  const long long nin = (long long)L.Vh << lgin, nout = (long long)L.Vh << lgout;
  const FieldRef& xs = p ? xo : xe;   // same parity as the output site
  const FieldRef& xn = p ? xe : xo;   // neighbours
  float acc[24];
#pragma unroll
  for (int m = 0; m < 24; ++m) acc[m] = 0.f;
  for (int i = 0; i < CI; ++i) {
    if (live && j < 9) {
      float v[24];
      if (j == 0) {
        SIO<P>::load(seg_ptr<P>(xs, L), seg_norm(xs, L), nin, ((long long)site << lgin) + i, v);
#pragma unroll
        for (int m = 0; m < 24; ++m) Z[s][0][m] = v[m];
      } else {
        const int d = j - 1;  // term 1 + 2mu: forward transport (link d = 2mu); 2 + 2mu: backward (d = 2mu + 1)
        SIO<P>::load(seg_ptr<P>(xn, L), seg_norm(xn, L), nin, ((long long)snb[d * NS + s] << lgin) + i, v);
        float z[24];
        colour_mul(su + (d * NS + s) * 18, v, z, (d & 1) != 0);
#pragma unroll
        for (int m = 0; m < 24; ++m) Z[s][j][m] = z[m];
        gamma_apply_rt(d >> 1, z, &Zg[s][j][0]);
      }
    }
    __syncthreads();
    if (live && j < CO) {
      const float2* w = W + ((size_t)j * CI + i);  // W[t][b][o][i] at ((t*4 + b)*CO + o)*CI + i
      const size_t tb = (size_t)CO * CI;
      {
        const float2 w0 = w[0], w1 = w[tb];
        const float2 cu = make_float2(w0.x + w1.x, w0.y + w1.y), cd = make_float2(w0.x - w1.x, w0.y - w1.y);
#pragma unroll
        for (int m = 0; m < 12; ++m) {
          const float2 z = make_float2(Z[s][0][2 * m], Z[s][0][2 * m + 1]);
          const float2 r = cmul(m < 6 ? cu : cd, z);
          acc[2 * m] += r.x;
          acc[2 * m + 1] += r.y;
        }
      }
      for (int t = 1; t < 9; ++t) {
        const float2 w0 = w[(4 * t + 0) * tb], w1 = w[(4 * t + 1) * tb], w2 = w[(4 * t + 2) * tb], w3 = w[(4 * t + 3) * tb];
        const float2 cu = make_float2(w0.x + w2.x, w0.y + w2.y), cd = make_float2(w0.x - w2.x, w0.y - w2.y);
        const float2 eu = make_float2(w1.x + w3.x, w1.y + w3.y), ed = make_float2(w1.x - w3.x, w1.y - w3.y);
#pragma unroll
        for (int m = 0; m < 12; ++m) {
          const float2 z = make_float2(Z[s][t][2 * m], Z[s][t][2 * m + 1]);
          const float2 zg = make_float2(Zg[s][t][2 * m], Zg[s][t][2 * m + 1]);
          const float2 r1 = cmul(m < 6 ? cu : cd, z), r2 = cmul(m < 6 ? eu : ed, zg);
          acc[2 * m] += r1.x + r2.x;
          acc[2 * m + 1] += r1.y + r2.y;
        }
      }
    }
    __syncthreads();
  }
  if (live && j < CO) SIO<P>::store(seg_ptr_w<P>(y, L), seg_norm(y, L), nout, ((long long)site << lgout) + j, acc);
}

// ------------------------------------------------------------ input gradient
// gx_i(x) = sum_o sum_b conj(W[0][b][o][i]) L_b g_o(x)
//         + sum_mu [ U_mu(x-mu)^+ m_f(x-mu) + U_mu(x) m_b(x+mu) ],
// m_{f,b}(y) = sum_o sum_b conj(W[1+2mu or 2+2mu][b][o][i]) H_b^+ g_o(y),
// H_b^+ = {1, g_mu, g5, -g5 g_mu}.
template <int P, int G>
__global__ void __launch_bounds__(256) nn_bwdx_kernel(LatDesc L, int p, FieldRef ge, FieldRef go, FieldRef gx,
                                                      const void* __restrict__ g32, const float2* __restrict__ W, int CI,
                                                      int CO, int lgin, int lgout) {
  extern __shared__ __align__(16) float sh[];
  float* su = sh;                              // [8][NS][18]
  int* snb = (int*)(su + 8 * NS * 18);         // [8][NS]
  float* Gs = (float*)(snb + 8 * NS);          // [NS][16][24]
  float* Gg = Gs + NS * 16 * 24;               // [NS][16][24]
  const int site0 = blockIdx.x * NS;
  stage_links<G>(L, p, site0, NS, gauge_seg<G>(g32, L), su, snb);
  __syncthreads();
  const int s = threadIdx.x >> 4, j = threadIdx.x & 15;
  const int site = site0 + s;
  const bool live = site < L.Vh;
  const long long nin = (long long)L.Vh << lgin, nout = (long long)L.Vh << lgout;
  const size_t tb = (size_t)CO * CI;
  float acc[24];
#pragma unroll
  for (int m = 0; m < 24; ++m) acc[m] = 0.f;
  for (int t = 0; t < 9; ++t) {
    // term t = 1 + 2mu gathers g at x - mu (neighbour d = 2mu + 1), term 2 + 2mu at x + mu (d = 2mu)
    const int mu = (t - 1) >> 1;
    const int d = t == 0 ? -1 : ((t & 1) ? 2 * mu + 1 : 2 * mu);
    if (live && j < CO) {
      float v[24];
      if (t == 0) {
        const FieldRef& gs = p ? go : ge;
        SIO<P>::load(seg_ptr<P>(gs, L), seg_norm(gs, L), nout, ((long long)site << lgout) + j, v);
      } else {
        const FieldRef& gn = p ? ge : go;
        SIO<P>::load(seg_ptr<P>(gn, L), seg_norm(gn, L), nout, ((long long)snb[d * NS + s] << lgout) + j, v);
        gamma_apply_rt(mu, v, Gg + (s * 16 + j) * 24);
      }
#pragma unroll
      for (int m = 0; m < 24; ++m) Gs[(s * 16 + j) * 24 + m] = v[m];
    }
    __syncthreads();
    if (live && j < CI) {
      float mm[24];
#pragma unroll
      for (int m = 0; m < 24; ++m) mm[m] = 0.f;
      for (int o = 0; o < CO; ++o) {
        const float2* w = W + ((size_t)o * CI + j);
        const float* gv = Gs + (s * 16 + o) * 24;
        if (t == 0) {
          const float2 w0 = w[0], w1 = w[tb];
          const float2 cu = make_float2(w0.x + w1.x, w0.y + w1.y), cd = make_float2(w0.x - w1.x, w0.y - w1.y);
#pragma unroll
          for (int m = 0; m < 12; ++m) {
            const float2 r = cmulc(m < 6 ? cu : cd, make_float2(gv[2 * m], gv[2 * m + 1]));
            mm[2 * m] += r.x;
            mm[2 * m + 1] += r.y;
          }
        } else {
          const float* gg = Gg + (s * 16 + o) * 24;
          const float2 w0 = w[(4 * t + 0) * tb], w1 = w[(4 * t + 1) * tb], w2 = w[(4 * t + 2) * tb], w3 = w[(4 * t + 3) * tb];
          // conj coefficients: up (c0 + c2), (c1 - c3); down (c0 - c2), (c1 + c3)
          const float2 cu = make_float2(w0.x + w2.x, w0.y + w2.y), cd = make_float2(w0.x - w2.x, w0.y - w2.y);
          const float2 eu = make_float2(w1.x - w3.x, w1.y - w3.y), ed = make_float2(w1.x + w3.x, w1.y + w3.y);
#pragma unroll
          for (int m = 0; m < 12; ++m) {
            const float2 r1 = cmulc(m < 6 ? cu : cd, make_float2(gv[2 * m], gv[2 * m + 1]));
            const float2 r2 = cmulc(m < 6 ? eu : ed, make_float2(gg[2 * m], gg[2 * m + 1]));
            mm[2 * m] += r1.x + r2.x;
            mm[2 * m + 1] += r1.y + r2.y;
          }
        }
      }
      if (t == 0) {
#pragma unroll
        for (int m = 0; m < 24; ++m) acc[m] += mm[m];
      } else {
        // t = 1 + 2mu: U_mu(x-mu)^+ (link d = 2mu + 1, adjoint); t = 2 + 2mu: U_mu(x) (link d = 2mu)
        float z[24];
        colour_mul(su + (d * NS + s) * 18, mm, z, (t & 1) != 0);
#pragma unroll
        for (int m = 0; m < 24; ++m) acc[m] += z[m];
      }
    }
    __syncthreads();
  }
  if (live && j < CI) SIO<P>::store(seg_ptr_w<P>(gx, L), seg_norm(gx, L), nin, ((long long)site << lgin) + j, acc);
}

// ----------------------------------------------------------- weight gradient
// grad W[t][b][o][i] = 2 sum_x <H_b Z_{t,i}(x), g_o(x)>, Z the transported inputs of
// the forward pass.  Persistent CTAs over tiles of NW sites; thread (o, i) keeps the
// 34 sums of its weight pair in registers and adds them to this CTA's slot of the
// partial buffer (deterministic: one writer per slot, launches in stream order).
constexpr int NW = 4;

template <int P, int G>
__global__ void __launch_bounds__(256) nn_bwdw_kernel(LatDesc L, int p, FieldRef xe, FieldRef xo, FieldRef gp,
                                                      const void* __restrict__ g32, int CI, int CO, int lgin, int lgout,
                                                      float2* __restrict__ partial, int ntile) {
  extern __shared__ __align__(16) float sh[];
  float* su = sh;                         // [8][NW][18]
  int* snb = (int*)(su + 8 * NW * 18);    // [8][NW]
  float* Z = (float*)(snb + 8 * NW);      // [NW][9][16][24]
  float* Zg = Z + NW * 9 * 16 * 24;       // [NW][9][16][24]
  float* Gs = Zg + NW * 9 * 16 * 24;      // [NW][16][24]
  const int o = threadIdx.x >> 4, i = threadIdx.x & 15;
  const bool mine = o < CO && i < CI;
  const long long nin = (long long)L.Vh << lgin, nout = (long long)L.Vh << lgout;
  const FieldRef& xs = p ? xo : xe;
  const FieldRef& xn = p ? xe : xo;
  const void* gb = gauge_seg<G>(g32, L);
  float2 a[34];
#pragma unroll
  for (int k = 0; k < 34; ++k) a[k] = make_float2(0.f, 0.f);
  for (int tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int site0 = tile * NW;
    __syncthreads();
    stage_links<G>(L, p, site0, NW, gb, su, snb);
    __syncthreads();
    // transported inputs of every channel: task (s, t, c)
    for (int task = threadIdx.x; task < NW * 9 * CI; task += blockDim.x) {
      const int c = task % CI, t = (task / CI) % 9, s = task / (CI * 9);
      const int site = site0 + s;
      float* zd = Z + ((s * 9 + t) * 16 + c) * 24;
      if (site >= L.Vh) {
        for (int m = 0; m < 24; ++m) zd[m] = 0.f;
        continue;
      }
      float v[24];
      if (t == 0) {
        SIO<P>::load(seg_ptr<P>(xs, L), seg_norm(xs, L), nin, ((long long)site << lgin) + c, v);
        for (int m = 0; m < 24; ++m) zd[m] = v[m];
      } else {
        const int d = t - 1;
        SIO<P>::load(seg_ptr<P>(xn, L), seg_norm(xn, L), nin, ((long long)snb[d * NW + s] << lgin) + c, v);
        colour_mul(su + (d * NW + s) * 18, v, zd, (d & 1) != 0);
        gamma_apply_rt(d >> 1, zd, Zg + ((s * 9 + t) * 16 + c) * 24);
      }
    }
    for (int task = threadIdx.x; task < NW * CO; task += blockDim.x) {
      const int c = task % CO, s = task / CO;
      const int site = site0 + s;
      float* gd = Gs + (s * 16 + c) * 24;
      if (site >= L.Vh) {
        for (int m = 0; m < 24; ++m) gd[m] = 0.f;
        continue;
      }
      float v[24];
      SIO<P>::load(seg_ptr<P>(gp, L), seg_norm(gp, L), nout, ((long long)site << lgout) + c, v);
      for (int m = 0; m < 24; ++m) gd[m] = v[m];
    }
    __syncthreads();
    if (mine) {
      for (int s = 0; s < NW; ++s) {
        const float* g = Gs + (s * 16 + o) * 24;
        for (int t = 0; t < 9; ++t) {
          const float* z = Z + ((s * 9 + t) * 16 + i) * 24;
          float2 au = make_float2(0.f, 0.f), ad = au, bu = au, bd = au;
#pragma unroll
          for (int m = 0; m < 12; ++m) {
            const float2 gm = make_float2(g[2 * m], g[2 * m + 1]);
            const float2 r = cmulc(make_float2(z[2 * m], z[2 * m + 1]), gm);
            if (m < 6) { au.x += r.x; au.y += r.y; } else { ad.x += r.x; ad.y += r.y; }
          }
          if (t == 0) {
            a[0].x += au.x + ad.x; a[0].y += au.y + ad.y;
            a[1].x += au.x - ad.x; a[1].y += au.y - ad.y;
          } else {
            const float* zg = Zg + ((s * 9 + t) * 16 + i) * 24;
#pragma unroll
            for (int m = 0; m < 12; ++m) {
              const float2 gm = make_float2(g[2 * m], g[2 * m + 1]);
              const float2 r = cmulc(make_float2(zg[2 * m], zg[2 * m + 1]), gm);
              if (m < 6) { bu.x += r.x; bu.y += r.y; } else { bd.x += r.x; bd.y += r.y; }
            }
            const int k = 2 + 4 * (t - 1);
            a[k + 0].x += au.x + ad.x; a[k + 0].y += au.y + ad.y;  // 1
            a[k + 1].x += bu.x + bd.x; a[k + 1].y += bu.y + bd.y;  // g_mu
            a[k + 2].x += au.x - ad.x; a[k + 2].y += au.y - ad.y;  // g5
            a[k + 3].x += bu.x - bd.x; a[k + 3].y += bu.y - bd.y;  // g5 g_mu
          }
        }
      }
    }
  }
  if (mine) {
    const size_t nW = (size_t)36 * CO * CI;
    float2* dst = partial + (size_t)blockIdx.x * nW;
    auto put = [&](int t, int b, float2 v) {
      float2& q = dst[((size_t)(t * 4 + b) * CO + o) * CI + i];
      q.x += 2.f * v.x;
      q.y += 2.f * v.y;
    };
    put(0, 0, a[0]);
    put(0, 1, a[1]);
    for (int t = 1; t < 9; ++t)
      for (int b = 0; b < 4; ++b) put(t, b, a[2 + 4 * (t - 1) + b]);
  }
}

__global__ void nn_wsum_kernel(const float2* __restrict__ partial, int nslice, size_t nW, float2* __restrict__ grad) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nW) return;
  double re = 0.0, im = 0.0;
  for (int sl = 0; sl < nslice; ++sl) {
    const float2 v = partial[(size_t)sl * nW + k];
    re += v.x;
    im += v.y;
  }
  grad[k] = make_float2((float)re, (float)im);
}

// g = (y - s) * inv_ns[0] (output gradient of |y - s|^2 / |s|^2), partial |y - s|^2
template <int P>
__global__ void nn_lossgrad_kernel(LatDesc L, FieldRef y, FieldRef s, FieldRef g, const double* __restrict__ inv_ns,
                                   double* partial, int pstride) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double red = 0.0;
  if (j < L.Vh) {
    float yv[24], sv[24];
    SIO<P>::load(seg_ptr<P>(y, L), seg_norm(y, L), L.Vh, j, yv);
    SIO<P32>::load(seg_ptr<P32>(s, L), nullptr, L.Vh, j, sv);
    const float sc = (float)inv_ns[0];
#pragma unroll
    for (int m = 0; m < 24; ++m) {
      const float d = yv[m] - sv[m];
      red += (double)d * (double)d;
      yv[m] = d * sc;
    }
    SIO<P>::store(seg_ptr_w<P>(g, L), seg_norm(g, L), L.Vh, j, yv);
  }
  block_reduce_cols(red, 1, partial, pstride);
}

__global__ void nn_adam_kernel(float2* W, const float2* __restrict__ grad, float2* m, float2* v, size_t n, float lr, float b1,
                               float b2, float eps, float c1, float c2, float gscale) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float2 g = make_float2(grad[k].x * gscale, grad[k].y * gscale);
  float2 mk = m[k], vk = v[k], w = W[k];
  mk.x = b1 * mk.x + (1.f - b1) * g.x;
  mk.y = b1 * mk.y + (1.f - b1) * g.y;
  vk.x = b2 * vk.x + (1.f - b2) * g.x * g.x;
  vk.y = b2 * vk.y + (1.f - b2) * g.y * g.y;
  w.x -= lr * (mk.x / c1) / (sqrtf(vk.x / c2) + eps);
  w.y -= lr * (mk.y / c1) / (sqrtf(vk.y / c2) + eps);
  m[k] = mk;
  v[k] = vk;
  W[k] = w;
}

// One column of a multi-column parity field to one column of another (the
// network's one-channel input and output against a block of right-hand sides).
template <int PD, int PS>
__global__ void copy_col_kernel(LatDesc L, FieldRef dst, int lgd, int cd, FieldRef src, int lgs, int cs) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.Vh) return;
  const long long nd = (long long)L.Vh << lgd, ns = (long long)L.Vh << lgs;
  typename SIO<PS>::real v[24];
  SIO<PS>::load(seg_ptr<PS>(src, L), seg_norm(src, L), ns, (i << lgs) + cs, v);
  typename SIO<PD>::real w[24];
#pragma unroll
  for (int m = 0; m < 24; ++m) w[m] = (typename SIO<PD>::real)v[m];
  SIO<PD>::store(seg_ptr_w<PD>(dst, L), seg_norm(dst, L), nd, (i << lgd) + cd, w);
}


// ------------------------------------------------ forward on the tensor cores
// bfloat16 activations: the channel mixing of a layer is a dense contraction,
// for each spin half h and spin-colour component c6 of that half
//   Y_(h,c6)[site][o] = sum_(t, i, kind) F_(t,i,kind)(site, h, c6) C_(h,t,kind)[o][i],
// F the transported inputs (kind 0: U x_i, kind 1: g_mu U x_i) and C the weight
// combinations of the spin factors on that half (W0 +- W2, W1 +- W3; +- = g5).
// As real GEMMs: M = 128 sites of one parity per CTA, N = 32 (16 channels x re/im),
// K = 64 per (term, kind) chunk (16 channels x re/im x re/im of F folded into B).
// Each chunk: 256 threads (two per site) transport and write 12 bf16 A tiles (one per (h, c6)) in
// the no-swizzle K-major core-matrix layout; one thread issues 24 tcgen05.mma
// (M128 N32 K16, FP32 accumulators in TMEM: 12 x 32 columns), commits to an
// mbarrier, and the CTA waits (bounded) before the next chunk overwrites the tiles.
// B (the weights) is laid out once per layer by nn_tc_prep_kernel.
constexpr int TC_M = 128;
constexpr int TC_ATILE = TC_M * 32 * 2;  // bytes of one A tile (128 rows x 32 bf16)
constexpr int TC_BCHUNK = 32 * 32 * 2;   // bytes of one B chunk (32 rows x 32 bf16)
constexpr int TC_SMEM = 12 * TC_ATILE + 2 * TC_BCHUNK + 64;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle, K-major; LBO = 128 B between the two
// 8 x 16 B core matrices adjacent in K, SBO = 512 B between 8-row groups
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)(128 >> 4) << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// byte offset of element (row r, k) of a 32-wide K tile
__device__ __forceinline__ int tc_off(int r, int k) { return (r >> 3) * 512 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2; }

// B chunks of one layer: [h 2][t 9][kind 2] x (32 n x 32 k), n = 2 o + part_y, k = 2 i + part_F
__global__ void nn_tc_prep_kernel(const float2* __restrict__ W, int CI, int CO, __nv_bfloat16* __restrict__ Bc) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 36 * 1024) return;
  const int chunk = e >> 10, w = e & 1023;
  const int n = w >> 5, k = w & 31;
  const int h = chunk / 18, t = (chunk / 2) % 9, kind = chunk & 1;
  const int o = n >> 1, py = n & 1, i = k >> 1, pf = k & 1;
  float cr = 0.f, ci = 0.f;
  if (o < CO && i < CI && !(t == 0 && kind == 1)) {
    const size_t tb = (size_t)CO * CI;
    const float sg = h ? -1.f : 1.f;
    float2 a, b;
    if (t == 0) {
      a = W[(size_t)o * CI + i];
      b = W[tb + (size_t)o * CI + i];
    } else {
      a = W[(4 * t + kind) * tb + (size_t)o * CI + i];
      b = W[(4 * t + kind + 2) * tb + (size_t)o * CI + i];
    }
    cr = a.x + sg * b.x;
    ci = a.y + sg * b.y;
  }
  // y_re += c_re F_re - c_im F_im ; y_im += c_im F_re + c_re F_im
  const float v = py == 0 ? (pf == 0 ? cr : -ci) : (pf == 0 ? ci : cr);
  Bc[(size_t)chunk * 1024 + tc_off(n, k) / 2] = __float2bfloat16_rn(v);
}

// Weights of the adjoint layer, so that the tensor-core forward computes the input
// gradient (the adjoint N^+ of a layer).  The layer sums W[t][b] H_b T_t x over terms t
// (T_0 = 1, T_{1+2mu} = U_mu(x) x(x+mu), T_{2+2mu} = U_mu(x-mu)^+ x(x-mu)) and spin factors
// H_b; the channel mixing, the spin factor and the colour transport act on different
// indices and commute, and T_{1+2mu}^+ = T_{2+2mu}, so the adjoint is a layer of the same
// form from C_out to C_in channels with
//   Wa[t][b][i][o] = s_b conj(W[t'][b][o][i]),  t' = t with the two hops of each mu swapped,
// s_b = -1 for H_3 = g5 g_mu (its adjoint is -g5 g_mu) and +1 otherwise (1, g5, g_mu are
// Hermitian).  Wa is [9][4][CI][CO].
__global__ void nn_adj_weights_kernel(const float2* __restrict__ W, int CI, int CO, float2* __restrict__ Wa) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 36 * CI * CO) return;
  const int o = e % CO, i = (e / CO) % CI, tb = e / (CO * CI);
  const int t = tb >> 2, b = tb & 3;
  const int ts = t == 0 ? 0 : ((t & 1) ? t + 1 : t - 1);
  const float2 w = W[((size_t)(4 * ts + b) * CO + o) * CI + i];
  const float sg = (t != 0 && b == 3) ? -1.f : 1.f;
  Wa[e] = make_float2(sg * w.x, -sg * w.y);
}

// 256 threads: thread tid transports channels 8 (tid >> 7) .. 8 (tid >> 7) + 7 of site
// tid & 127; in the epilogue warps w and w + 4 share TMEM lanes 32 (w & 3) .. and
// write output channels 0..7 and 8..15 of those sites.
template <int G>
__global__ void __launch_bounds__(256, 1) nn_fwd_tc_kernel(LatDesc L, int p, FieldRef xe, FieldRef xo, FieldRef y,
                                                           const void* __restrict__ g32,
                                                           const __nv_bfloat16* __restrict__ Bc, int CI, int CO,
                                                           int lgin, int lgout, int* err) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  unsigned char* sA = tc_smem;                          // 12 A tiles
  unsigned char* sB = tc_smem + 12 * TC_ATILE;          // 2 B chunks (halves)
  uint64_t* mbar = (uint64_t*)(sB + 2 * TC_BCHUNK);
  uint32_t* tslot = (uint32_t*)(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid & (TC_M - 1), half = tid >> 7;
  const int site = blockIdx.x * TC_M + row;
  const bool live = site < L.Vh;
  const long long nin = (long long)L.Vh << lgin, nout = (long long)L.Vh << lgout;
  const FieldRef& xs = p ? xo : xe;
  const FieldRef& xn = p ? xe : xo;
  const void* gb = gauge_seg<G>(g32, L);
  int x = 0, yy = 0, z = 0, t = 0;
  if (live) cb_coords(L, site, p, x, yy, z, t);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  // M = 128, N = 32, A and B bf16 K-major, D FP32
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(32 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  bool ok = true;
  int chunk = 0;
  for (int term = 0; term < 9 && ok; ++term) {
    // this term's link and neighbour (terms 1 + 2 mu forward, 2 + 2 mu backward)
    float u[18];
    long long nbr = site;
    if (term > 0 && live) {
      const int d = term - 1, mu = d >> 1;
      const bool bwd = d & 1;
      int xn_ = x, yn = yy, zn = z, tn = t;
      bool crosses = false;
      if (mu == 0) xn_ = bwd ? (x == 0 ? L.X - 1 : x - 1) : (x + 1 == L.X ? 0 : x + 1);
      else if (mu == 1) yn = bwd ? (yy == 0 ? L.Y - 1 : yy - 1) : (yy + 1 == L.Y ? 0 : yy + 1);
      else if (mu == 2) zn = bwd ? (z == 0 ? L.Z - 1 : z - 1) : (z + 1 == L.Z ? 0 : z + 1);
      else {
        crosses = bwd ? (t == 0) : (t + 1 == L.T);
        tn = bwd ? (t == 0 ? L.T - 1 : t - 1) : (t + 1 == L.T ? 0 : t + 1);
      }
      nbr = lex_of(L, xn_, yn, zn, tn) >> 1;
      GIO<G>::load(gb, L.Vh, bwd ? 1 - p : p, mu, bwd ? (int)nbr : site, u);
      const float f = crosses ? (float)L.tbc : 1.f;
#pragma unroll
      for (int e = 0; e < 18; ++e) u[e] *= f;
    }
    for (int kind = 0; kind < (term == 0 ? 1 : 2) && ok; ++kind, ++chunk) {
      if (chunk > 0) {  // the previous chunk's MMAs must have read the tiles
        int done = 0;
        for (int it = 0; it < (1 << 24) && !done; ++it) {
          uint32_t r;
          asm volatile(
              "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
              : "=r"(r)
              : "r"(smem_u32(mbar)), "r"((uint32_t)((chunk - 1) & 1)));
          done = r;
        }
        // one decision for the whole CTA (threads start polling at different times): if
        // any thread gave up, every thread leaves the chunk loop before its next barrier
        if (!__syncthreads_and(done)) {
          ok = false;
          if (tid == 0) atomicExch(err, 1);
          break;
        }
      }
      // A tiles: this thread's row, its 8 channels
      for (int i = 8 * half; i < 8 * half + 8; ++i) {
        float v[24];
        if (live && i < CI) {
          if (term == 0) {
            SIO<PBF>::load(seg_ptr<PBF>(xs, L), nullptr, nin, ((long long)site << lgin) + i, v);
          } else {
            float w0[24];
            const int d = term - 1;
            SIO<PBF>::load(seg_ptr<PBF>(xn, L), nullptr, nin, (nbr << lgin) + i, w0);
            colour_mul(u, w0, v, (d & 1) != 0);
            if (kind == 1) {
              float g[24];
              gamma_apply_rt(d >> 1, v, g);
#pragma unroll
              for (int m = 0; m < 24; ++m) v[m] = g[m];
            }
          }
        } else {
#pragma unroll
          for (int m = 0; m < 24; ++m) v[m] = 0.f;
        }
#pragma unroll
        for (int m = 0; m < 12; ++m)
          *(__nv_bfloat162*)(sA + m * TC_ATILE + tc_off(row, 2 * i)) = __floats2bfloat162_rn(v[2 * m], v[2 * m + 1]);
      }
      // B chunks of both halves for (term, kind)
      for (int e = tid; e < 2 * TC_BCHUNK / 16; e += blockDim.x) {
        const int h = e / (TC_BCHUNK / 16), q = e % (TC_BCHUNK / 16);
        const uint4* src = (const uint4*)(Bc + (size_t)((h * 9 + term) * 2 + kind) * 1024);
        ((uint4*)(sB + h * TC_BCHUNK))[q] = __ldg(src + q);
      }
      asm volatile("fence.proxy.async.shared::cta;");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (tid == 0) {
#pragma unroll 1
        for (int g = 0; g < 12; ++g)
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            const uint64_t da = tc_desc(smem_u32(sA + g * TC_ATILE + ks * 256));
            const uint64_t db = tc_desc(smem_u32(sB + (g / 6) * TC_BCHUNK + ks * 256));
            const uint32_t acc = (chunk > 0 || ks > 0) ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n\t}\n" ::"r"(tmem + (uint32_t)(g * 32)),
                "l"(da), "l"(db), "r"(idesc), "r"(acc));
          }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar)));
      }
    }
  }
  // wait for the last chunk's MMAs (also on an error path: nothing may be in flight at dealloc)
  {
    int done = 0;
    for (int it = 0; it < (1 << 24) && !done; ++it) {
      uint32_t r;
      asm volatile(
          "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
          : "=r"(r)
          : "r"(smem_u32(mbar)), "r"((uint32_t)((chunk - 1) & 1)));
      done = r;
    }
    if (!__syncthreads_and(done)) {  // the same decision in every thread
      ok = false;
      if (tid == 0) atomicExch(err, 1);
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    // epilogue: this thread's site = TMEM lane; chunk kk of the bf16 output holds components
    // 4 kk .. 4 kk + 3; this warp reads the 16 columns (8 channels x re/im) of its half
    const uint32_t lane_base = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(16 * half);
    for (int kk = 0; kk < 3; ++kk) {
      uint32_t r[4][16];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t ta = lane_base + (uint32_t)((4 * kk + q) * 32);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[q][0]), "=r"(r[q][1]), "=r"(r[q][2]), "=r"(r[q][3]), "=r"(r[q][4]), "=r"(r[q][5]), "=r"(r[q][6]),
              "=r"(r[q][7]), "=r"(r[q][8]), "=r"(r[q][9]), "=r"(r[q][10]), "=r"(r[q][11]), "=r"(r[q][12]),
              "=r"(r[q][13]), "=r"(r[q][14]), "=r"(r[q][15])
            : "r"(ta));
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (live) {
        uint4* out = (uint4*)seg_ptr_w<PBF>(y, L);
#pragma unroll
        for (int oo = 0; oo < 8; ++oo) {
          const int o = 8 * half + oo;
          if (o < CO) {
            uint4 c;
            __nv_bfloat162* hh = reinterpret_cast<__nv_bfloat162*>(&c);
#pragma unroll
            for (int q = 0; q < 4; ++q)
              hh[q] = __floats2bfloat162_rn(__uint_as_float(r[q][2 * oo]), __uint_as_float(r[q][2 * oo + 1]));
            out[kk * nout + ((long long)site << lgout) + o] = c;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// ------------------------------------------- weight gradient on the tensor cores
// bfloat16 activations.  With F_(t,i,kind)(site, h, c6) the transported inputs of the
// forward pass (kind 0: Z = T_t x_i, kind 1: g_mu Z; spin half h, spin-colour component c6
// of that half) and G(site, h, c6)[o] the output gradient, the gradient of the weight
// combination C_(h,t,kind)[o][i] of the forward kernel is
//   dC_h[o][i] = sum_(site, c6) conj(F_(t,i,kind)(site, h, c6)) G(site, h, c6)[o],
// and grad W[t][kind] = 2 (dC_0 + dC_1), grad W[t][kind + 2] = 2 (dC_0 - dC_1) (term 0: its
// two spin factors 1 and g5 are b = 0 and 1), the sums of the CUDA-core kernel above.  As
// real GEMMs with the sites as the reduction dimension: for each spin half h and group of
// two terms (term 0 alone), D_h[(term, kind, i, re/im of F)][(o, re/im of G)] (M = 128,
// N = 32) accumulates A_(h,c6) B_(h,c6)^T over c6 and over the CTA's sites, K = 32 sites
// per tile, bf16 operands in the forward kernel's K-major core-matrix layout.  Persistent
// CTAs (one per partial slot) keep the ten accumulators (5 groups x 2 halves, 320 TMEM
// columns) in tensor memory for the whole launch and add them to their slot at the end.
// Each group: 256 threads (site lane & 31, input channels 2 (tid >> 5), + 1) transport and
// write the A tiles, one thread issues 24 tcgen05.mma, and the CTA waits (bounded) for them
// before the tiles are overwritten.
constexpr int TW_S = 32;                   // sites per tile
constexpr int TW_ATILE = 128 * TW_S * 2;   // A tile: 128 rows x 32 sites, bf16
constexpr int TW_BTILE = 32 * TW_S * 2;    // B tile: 32 rows x 32 sites
constexpr int TW_SMEM = 12 * TW_ATILE + 12 * TW_BTILE + 8 * TW_S * 18 * 4 + 8 * TW_S * 4 + 64;

__device__ __forceinline__ void tc_put_bf16(unsigned char* tile, int r, int k, float v) {
  *(__nv_bfloat16*)(tile + tc_off(r, k)) = __float2bfloat16_rn(v);
}

// Bounded wait for the commit with the given parity; one decision for the whole CTA.
__device__ __forceinline__ bool tc_wait_all(uint64_t* mbar, uint32_t parity) {
  int done = 0;
  for (int it = 0; it < (1 << 24) && !done; ++it) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"(smem_u32(mbar)), "r"(parity));
    done = r;
  }
  return __syncthreads_and(done) != 0;
}

template <int G>
__global__ void __launch_bounds__(256, 1) nn_bwdw_tc_kernel(LatDesc L, int p, FieldRef xe, FieldRef xo, FieldRef gp,
                                                            const void* __restrict__ g32, int CI, int CO, int lgin,
                                                            int lgout, float2* __restrict__ partial, int ntile,
                                                            int* err) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  unsigned char* sA = tc_smem;                      // 12 A tiles, one per (h, c6)
  unsigned char* sB = sA + 12 * TW_ATILE;           // 12 B tiles
  float* su = (float*)(sB + 12 * TW_BTILE);         // [8][TW_S][18] links
  int* snb = (int*)(su + 8 * TW_S * 18);            // [8][TW_S] neighbours
  uint64_t* mbar = (uint64_t*)(snb + 8 * TW_S);
  uint32_t* tslot = (uint32_t*)(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, s = tid & 31;
  const long long nin = (long long)L.Vh << lgin, nout = (long long)L.Vh << lgout;
  const FieldRef& xs = p ? xo : xe;
  const FieldRef& xn = p ? xe : xo;
  const void* gb = gauge_seg<G>(g32, L);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  // M = 128, N = 32, A and B bf16 K-major, D FP32
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(32 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  bool ok = true;
  int ncommit = 0;
  for (int tile = blockIdx.x; tile < ntile && ok; tile += gridDim.x) {
    const int site0 = tile * TW_S, site = site0 + s;
    const bool live = site < L.Vh;
    __syncthreads();  // the previous tile's threads are done with su / snb
    stage_links<G>(L, p, site0, TW_S, gb, su, snb);
    // B tiles: the output gradient of this thread's site, outputs 2 warp and 2 warp + 1
    for (int oo = 0; oo < 2; ++oo) {
      const int o = 2 * warp + oo;
      float v[24];
      if (live && o < CO) {
        SIO<PBF>::load(seg_ptr<PBF>(gp, L), nullptr, nout, ((long long)site << lgout) + o, v);
      } else {
#pragma unroll
        for (int m = 0; m < 24; ++m) v[m] = 0.f;
      }
#pragma unroll
      for (int m = 0; m < 12; ++m) {
        tc_put_bf16(sB + m * TW_BTILE, 2 * o, s, v[2 * m]);
        tc_put_bf16(sB + m * TW_BTILE, 2 * o + 1, s, v[2 * m + 1]);
      }
    }
    __syncthreads();  // links staged
    for (int g = 0; g < 5 && ok; ++g) {
      // A tiles: row ((tl * 2 + kind) * 16 + i) * 2 + re/im for term tl of the group
      for (int tl = 0; tl < 2; ++tl) {
        const int t = g == 0 ? (tl == 0 ? 0 : -1) : 2 * g - 1 + tl;
        for (int ii = 0; ii < 2; ++ii) {
          const int i = 2 * warp + ii;
          float z[24], zg[24];
          if (t >= 0 && live && i < CI) {
            if (t == 0) {
              SIO<PBF>::load(seg_ptr<PBF>(xs, L), nullptr, nin, ((long long)site << lgin) + i, z);
#pragma unroll
              for (int m = 0; m < 24; ++m) zg[m] = 0.f;
            } else {
              const int d = t - 1;
              float v[24];
              SIO<PBF>::load(seg_ptr<PBF>(xn, L), nullptr, nin, ((long long)snb[d * TW_S + s] << lgin) + i, v);
              colour_mul(su + (d * TW_S + s) * 18, v, z, (d & 1) != 0);
              gamma_apply_rt(d >> 1, z, zg);
            }
          } else {
#pragma unroll
            for (int m = 0; m < 24; ++m) z[m] = zg[m] = 0.f;
          }
          const int r0 = ((tl * 2) * 16 + i) * 2, r1 = ((tl * 2 + 1) * 16 + i) * 2;
#pragma unroll
          for (int m = 0; m < 12; ++m) {
            unsigned char* a = sA + m * TW_ATILE;
            tc_put_bf16(a, r0, s, z[2 * m]);
            tc_put_bf16(a, r0 + 1, s, z[2 * m + 1]);
            tc_put_bf16(a, r1, s, zg[2 * m]);
            tc_put_bf16(a, r1 + 1, s, zg[2 * m + 1]);
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (tid == 0) {
        const bool first_tile = tile == (int)blockIdx.x;
#pragma unroll 1
        for (int m = 0; m < 12; ++m)
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            const uint64_t da = tc_desc(smem_u32(sA + m * TW_ATILE + ks * 256));
            const uint64_t db = tc_desc(smem_u32(sB + m * TW_BTILE + ks * 256));
            const uint32_t acc = (first_tile && (m % 6) == 0 && ks == 0) ? 0u : 1u;
            asm volatile(
                "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n\t}\n" ::"r"(
                    tmem + (uint32_t)((2 * g + m / 6) * 32)),
                "l"(da), "l"(db), "r"(idesc), "r"(acc));
          }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar)));
      }
      // the tiles are rewritten next: wait for these MMAs (every thread, one decision)
      if (!tc_wait_all(mbar, (uint32_t)(ncommit & 1))) {
        ok = false;
        if (tid == 0) atomicExch(err, 1);
      }
      ++ncommit;
      asm volatile("tcgen05.fence::after_thread_sync;");
    }
  }
  // an expired wait: give the MMAs in flight a second bounded wait before the release
  if (!ok && ncommit > 0) tc_wait_all(mbar, (uint32_t)((ncommit - 1) & 1));
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    // epilogue: thread = accumulator row r (TMEM lane), 16 columns (8 outputs x re/im of G)
    // of its warp's half; the partner row r ^ 1 (the other re/im of F) is the next lane
    const int half = warp >> 2, rowbase = 32 * (warp & 3);
    const int r = rowbase + (tid & 31);
    const int pf = r & 1, i = (r >> 1) & 15, kind = (r >> 5) & 1, tl = (r >> 6) & 1;
    const size_t nW = (size_t)36 * CO * CI;
    float2* dst = partial + (size_t)blockIdx.x * nW;
    for (int g = 0; g < 5; ++g) {
      uint32_t d[2][16];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t ta = tmem + ((uint32_t)rowbase << 16) + (uint32_t)((2 * g + h) * 32 + 16 * half);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(d[h][0]), "=r"(d[h][1]), "=r"(d[h][2]), "=r"(d[h][3]), "=r"(d[h][4]), "=r"(d[h][5]), "=r"(d[h][6]),
              "=r"(d[h][7]), "=r"(d[h][8]), "=r"(d[h][9]), "=r"(d[h][10]), "=r"(d[h][11]), "=r"(d[h][12]),
              "=r"(d[h][13]), "=r"(d[h][14]), "=r"(d[h][15])
            : "r"(ta));
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      const int t = g == 0 ? (tl == 0 ? 0 : -1) : 2 * g - 1 + tl;
      const bool row_ok = pf == 0 && t >= 0 && !(t == 0 && kind == 1) && i < CI;
      const int bs = t == 0 ? 0 : kind, bd = t == 0 ? 1 : kind + 2;
#pragma unroll
      for (int oo = 0; oo < 8; ++oo) {
        float2 dc[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float ar = __uint_as_float(d[h][2 * oo]), ai = __uint_as_float(d[h][2 * oo + 1]);
          const float br = __shfl_xor_sync(0xffffffffu, ar, 1), bi = __shfl_xor_sync(0xffffffffu, ai, 1);
          // own row F_re, partner row F_im: conj(F) G = (F_re G_re + F_im G_im) + i (F_re G_im - F_im G_re)
          dc[h] = make_float2(ar + bi, ai - br);
        }
        const int o = 8 * half + oo;
        if (row_ok && o < CO) {
          float2& qs = dst[((size_t)(t * 4 + bs) * CO + o) * CI + i];
          float2& qd = dst[((size_t)(t * 4 + bd) * CO + o) * CI + i];
          qs.x += 2.f * (dc[0].x + dc[1].x);
          qs.y += 2.f * (dc[0].y + dc[1].y);
          qd.x += 2.f * (dc[0].x - dc[1].x);
          qd.y += 2.f * (dc[0].y - dc[1].y);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

}  // namespace

namespace dl {

// Backward launches with more than the default 48 KB of dynamic shared memory: the
// attribute is set (and checked) before every launch.
template <int PP, int GG>
cudaError_t launch_bwdx(int grid, size_t smem, const LatDesc& L, int parity, FieldRef ge, FieldRef go, FieldRef gx,
                        const void* g32, const float2* W, int ci, int co, int lgin, int lgout, cudaStream_t st) {
  DL_CUDA_TRY(cudaFuncSetAttribute(nn_bwdx_kernel<PP, GG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  DL_COUNT();
  nn_bwdx_kernel<PP, GG><<<grid, 256, smem, st>>>(L, parity, ge, go, gx, g32, W, ci, co, lgin, lgout);
  return cudaGetLastError();
}

template <int PP, int GG>
cudaError_t launch_bwdw(int grid, size_t smem, const LatDesc& L, int parity, FieldRef xe, FieldRef xo, FieldRef gp,
                        const void* g32, int ci, int co, int lgin, int lgout, float2* partial, int ntile,
                        cudaStream_t st) {
  DL_CUDA_TRY(cudaFuncSetAttribute(nn_bwdw_kernel<PP, GG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  DL_COUNT();
  nn_bwdw_kernel<PP, GG><<<grid, 256, smem, st>>>(L, parity, xe, xo, gp, g32, ci, co, lgin, lgout, partial, ntile);
  return cudaGetLastError();
}

#define NN_DISPATCH(P, G, CALL)                                       \
  if (P == P32 && G == 12) { constexpr int PP = P32; constexpr int GG = G32R12; CALL; } \
  else if (P == P32 && G == 8) { constexpr int PP = P32; constexpr int GG = G32R8; CALL; } \
  else if (P == PBF && G == 12) { constexpr int PP = PBF; constexpr int GG = G32R12; CALL; } \
  else if (P == PBF && G == 8) { constexpr int PP = PBF; constexpr int GG = G32R8; CALL; } \
  else return cudaErrorInvalidValue;

cudaError_t nn_forward(const LatDesc& L, int prec, int grec, int parity, FieldRef xe, FieldRef xo, FieldRef y,
                       const void* g32, const float2* W, int ci, int co, int lgin, int lgout, cudaStream_t st) {
  if (ci > 16 || co > 16 || ci < 1 || co < 1) return cudaErrorInvalidValue;
  const int grid = (L.Vh + NS - 1) / NS;
  NN_DISPATCH(prec, grec, (DL_COUNT(), nn_fwd_kernel<PP, GG><<<grid, 256, 0, st>>>(L, parity, xe, xo, y, g32, W, ci, co, lgin, lgout)));
  return cudaGetLastError();
}

cudaError_t nn_backward_x(const LatDesc& L, int prec, int grec, int parity, FieldRef ge, FieldRef go, FieldRef gx,
                          const void* g32, const float2* W, int ci, int co, int lgin, int lgout, cudaStream_t st) {
  if (ci > 16 || co > 16 || ci < 1 || co < 1) return cudaErrorInvalidValue;
  const int grid = (L.Vh + NS - 1) / NS;
  const size_t smem = (size_t)8 * NS * 18 * 4 + 8 * NS * 4 + (size_t)2 * NS * 16 * 24 * 4;
  NN_DISPATCH(prec, grec, return (launch_bwdx<PP, GG>(grid, smem, L, parity, ge, go, gx, g32, W, ci, co, lgin, lgout, st)));
}

// partial: nslots x (36 * co * ci) complex, this parity's slots start at `partial`;
// the launch uses `slots` persistent CTAs.
cudaError_t nn_backward_w(const LatDesc& L, int prec, int grec, int parity, FieldRef xe, FieldRef xo, FieldRef gp,
                          const void* g32, int ci, int co, int lgin, int lgout, float2* partial, int slots,
                          cudaStream_t st) {
  if (ci > 16 || co > 16 || ci < 1 || co < 1) return cudaErrorInvalidValue;
  const int ntile = (L.Vh + NW - 1) / NW;
  const int grid = slots < ntile ? slots : ntile;
  const size_t smem = (size_t)8 * NW * 18 * 4 + 8 * NW * 4 + (size_t)2 * NW * 9 * 16 * 24 * 4 + (size_t)NW * 16 * 24 * 4;
  NN_DISPATCH(prec, grec,
              return (launch_bwdw<PP, GG>(grid, smem, L, parity, xe, xo, gp, g32, ci, co, lgin, lgout, partial, ntile, st)));
}

cudaError_t nn_backward_w_tc(const LatDesc& L, int grec, int parity, FieldRef xe, FieldRef xo, FieldRef gp,
                             const void* g32, int ci, int co, int lgin, int lgout, float2* partial, int slots, int* err,
                             cudaStream_t st) {
  if (ci > 16 || co > 16 || ci < 1 || co < 1 || slots < 1) return cudaErrorInvalidValue;
  const int ntile = (L.Vh + TW_S - 1) / TW_S;
  const int grid = slots < ntile ? slots : ntile;  // every CTA has at least one tile
  if (grid < 1) return cudaSuccess;
  if (grec == 12) {
    DL_CUDA_TRY(cudaFuncSetAttribute(nn_bwdw_tc_kernel<G32R12>, cudaFuncAttributeMaxDynamicSharedMemorySize, TW_SMEM));
    DL_COUNT();
    nn_bwdw_tc_kernel<G32R12><<<grid, 256, TW_SMEM, st>>>(L, parity, xe, xo, gp, g32, ci, co, lgin, lgout, partial,
                                                           ntile, err);
  } else if (grec == 8) {
    DL_CUDA_TRY(cudaFuncSetAttribute(nn_bwdw_tc_kernel<G32R8>, cudaFuncAttributeMaxDynamicSharedMemorySize, TW_SMEM));
    DL_COUNT();
    nn_bwdw_tc_kernel<G32R8><<<grid, 256, TW_SMEM, st>>>(L, parity, xe, xo, gp, g32, ci, co, lgin, lgout, partial,
                                                          ntile, err);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t nn_wsum(const float2* partial, int nslice, size_t nW, float2* grad, cudaStream_t st) {
  DL_COUNT();
  nn_wsum_kernel<<<(unsigned)((nW + 255) / 256), 256, 0, st>>>(partial, nslice, nW, grad);
  return cudaGetLastError();
}

cudaError_t nn_lossgrad(const Batch& B, int prec, FieldRef y, FieldRef s, FieldRef g, const double* inv_ns, double* partial,
                        cudaStream_t st) {
  const LatDesc& L = B.lat[0];
  const int grid = (L.Vh + 255) / 256;
  if (prec == P32) {
    DL_COUNT();
    nn_lossgrad_kernel<P32><<<grid, 256, 0, st>>>(L, y, s, g, inv_ns, partial, B.pstride);
  } else if (prec == PBF) {
    DL_COUNT();
    nn_lossgrad_kernel<PBF><<<grid, 256, 0, st>>>(L, y, s, g, inv_ns, partial, B.pstride);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t nn_adam(float2* W, const float2* grad, float2* m, float2* v, size_t n, float lr, float b1, float b2, float eps,
                    int step, float gscale, cudaStream_t st) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  DL_COUNT();
  nn_adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(W, grad, m, v, n, lr, b1, b2, eps, c1, c2, gscale);
  return cudaGetLastError();
}

cudaError_t copy_col(const LatDesc& L, int pd, int ps, FieldRef dst, int lgd, int cd, FieldRef src, int lgs, int cs,
                     cudaStream_t st) {
  const int grid = (L.Vh + 255) / 256;
#define CC(a, b)                                                                                      \
  if (pd == a && ps == b) {                                                                         \
    DL_COUNT();                                                                                     \
    copy_col_kernel<a, b><<<grid, 256, 0, st>>>(L, dst, lgd, cd, src, lgs, cs);                     \
    return cudaGetLastError();                                                                      \
  }
  CC(P32, P32) CC(P32, PBF) CC(PBF, P32) CC(P64, PBF) CC(PBF, P64) CC(P64, P32) CC(P32, P64) CC(P64, P64)
#undef CC
  return cudaErrorInvalidValue;
}

cudaError_t nn_tc_prep(const float2* W, int ci, int co, void* Bc, cudaStream_t st) {
  if (ci > 16 || co > 16 || ci < 1 || co < 1) return cudaErrorInvalidValue;
  DL_COUNT();
  nn_tc_prep_kernel<<<36 * 1024 / 256, 256, 0, st>>>(W, ci, co, (__nv_bfloat16*)Bc);
  return cudaGetLastError();
}

cudaError_t nn_adj_weights(const float2* W, int ci, int co, float2* Wa, cudaStream_t st) {
  if (ci > 16 || co > 16 || ci < 1 || co < 1) return cudaErrorInvalidValue;
  DL_COUNT();
  nn_adj_weights_kernel<<<(36 * ci * co + 255) / 256, 256, 0, st>>>(W, ci, co, Wa);
  return cudaGetLastError();
}

cudaError_t nn_forward_tc(const LatDesc& L, int grec, int parity, FieldRef xe, FieldRef xo, FieldRef y, const void* g32,
                          const void* Bc, int ci, int co, int lgin, int lgout, int* err, cudaStream_t st) {
  if (ci > 16 || co > 16 || ci < 1 || co < 1) return cudaErrorInvalidValue;
  const int grid = (L.Vh + TC_M - 1) / TC_M;
  if (grec == 12) {
    DL_CUDA_TRY(cudaFuncSetAttribute(nn_fwd_tc_kernel<G32R12>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
    DL_COUNT();
    nn_fwd_tc_kernel<G32R12><<<grid, 256, TC_SMEM, st>>>(L, parity, xe, xo, y, g32, (const __nv_bfloat16*)Bc, ci, co,
                                                          lgin, lgout, err);
  } else if (grec == 8) {
    DL_CUDA_TRY(cudaFuncSetAttribute(nn_fwd_tc_kernel<G32R8>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
    DL_COUNT();
    nn_fwd_tc_kernel<G32R8><<<grid, 256, TC_SMEM, st>>>(L, parity, xe, xo, y, g32, (const __nv_bfloat16*)Bc, ci, co,
                                                         lgin, lgout, err);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace dl
