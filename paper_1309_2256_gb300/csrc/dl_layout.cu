// Layout kernels: natural <-> even-odd device fields, gauge compression
// (reconstruct 18/12/8, App. A "Twisted mass fermion operator"), and the
// counter-based Z4 noise of the stochastic estimator (Sec. 2.1).
#include "dl_internal.cuh"
#include "dl_kernels.h"

namespace {

// Natural field (one lattice): complex [col][lex][12], dtype C128 (0) or C64 (1).
template <int P>
__global__ void pack_kernel(Batch B, int parity, FieldRef dst, const void* natural, int dtype) {
  const LatDesc& L = B.lat[0];
  const int npad = 1 << L.lognpad;
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nitems = (long long)L.Vh * npad;
  if (j >= nitems) return;
  const int col = (int)(j & (npad - 1));
  const int i = (int)(j >> L.lognpad);
  typename SIO<P>::real v[24];
  if (col < L.ncol) {
    int x, y, z, t;
    cb_coords(L, i, parity, x, y, z, t);
    const long long V = 2LL * L.Vh;
    const long long base = ((long long)col * V + lex_of(L, x, y, z, t)) * 12;
    if (dtype == 0) {
      const double2* src = (const double2*)natural + base;
#pragma unroll
      for (int m = 0; m < 12; ++m) {
        double2 c = src[m];
        v[2 * m] = (typename SIO<P>::real)c.x;
        v[2 * m + 1] = (typename SIO<P>::real)c.y;
      }
    } else {
      const float2* src = (const float2*)natural + base;
#pragma unroll
      for (int m = 0; m < 12; ++m) {
        float2 c = src[m];
        v[2 * m] = (typename SIO<P>::real)c.x;
        v[2 * m + 1] = (typename SIO<P>::real)c.y;
      }
    }
  } else {
#pragma unroll
    for (int m = 0; m < 24; ++m) v[m] = 0;
  }
  SIO<P>::store(seg_ptr_w<P>(dst, L), seg_norm(dst, L), nitems, j, v);
}

template <int P>
__global__ void unpack_kernel(Batch B, int parity, void* natural, FieldRef src, int dtype) {
  const LatDesc& L = B.lat[0];
  const int npad = 1 << L.lognpad;
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nitems = (long long)L.Vh * npad;
  if (j >= nitems) return;
  const int col = (int)(j & (npad - 1));
  if (col >= L.ncol) return;
  const int i = (int)(j >> L.lognpad);
  int x, y, z, t;
  cb_coords(L, i, parity, x, y, z, t);
  typename SIO<P>::real v[24];
  SIO<P>::load(seg_ptr<P>(src, L), seg_norm(src, L), nitems, j, v);
  const long long V = 2LL * L.Vh;
  const long long base = ((long long)col * V + lex_of(L, x, y, z, t)) * 12;
  if (dtype == 0) {
    double2* d = (double2*)natural + base;
#pragma unroll
    for (int m = 0; m < 12; ++m) d[m] = make_double2((double)v[2 * m], (double)v[2 * m + 1]);
  } else {
    float2* d = (float2*)natural + base;
#pragma unroll
    for (int m = 0; m < 12; ++m) d[m] = make_float2((float)v[2 * m], (float)v[2 * m + 1]);
  }
}

// splitmix64 (Steele, Lea & Flood 2014): state = seed + (n + 1) * golden, then
// the published output mix.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed, unsigned long long n) {
  unsigned long long z = seed + (n + 1ULL) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Entry (noise r, lex, spin a, colour c) from bits 0 and 1 of
// splitmix64(seed, (r*V + lex)*12 + 3a + c): (s1 + i s2)/sqrt(2) with
// s = 1 - 2*bit, or {1, i, -1, -i}[bit0 + 2*bit1] for the quadrant form.
// Sites on time slices outside S are zero (time-diluted sources, Sec. 2.3).
template <int P>
__global__ void noise_kernel(Batch B, int parity, FieldRef dst, unsigned long long seed, unsigned long long first,
                             int quadrant, Slices S) {
  const int l = find_lat(B, blockIdx.x);
  const LatDesc& L = B.lat[l];
  const int npad = 1 << L.lognpad;
  const long long j = (long long)(blockIdx.x - B.blk_begin[l]) * blockDim.x + threadIdx.x;
  const long long nitems = (long long)L.Vh * npad;
  if (j >= nitems) return;
  const int col = (int)(j & (npad - 1));
  const int i = (int)(j >> L.lognpad);
  typename SIO<P>::real v[24];
  int x, y, z, t;
  cb_coords(L, i, parity, x, y, z, t);
  if (col < L.ncol && slice_index(S, t) >= 0) {
    const unsigned long long V = 2ULL * (unsigned long long)L.Vh;
    const unsigned long long r = first + (unsigned long long)L.noise_base + (unsigned long long)col;
    const unsigned long long n0 = (r * V + (unsigned long long)lex_of(L, x, y, z, t)) * 12ULL;
    typedef typename SIO<P>::real R;
    const R h = (R)(1.0 / sqrt(2.0));  // folded at compile time; entries are selected, not computed
#pragma unroll
    for (int m = 0; m < 12; ++m) {
      unsigned long long w = splitmix64(seed, n0 + (unsigned long long)m);
      int b0 = (int)(w & 1ULL), b1 = (int)((w >> 1) & 1ULL);
      R re, im;
      if (quadrant) {
        int qd = b0 + 2 * b1;
        re = (qd == 0) ? (R)1 : (qd == 2 ? (R)-1 : (R)0);
        im = (qd == 1) ? (R)1 : (qd == 3 ? (R)-1 : (R)0);
      } else {
        re = b0 ? -h : h;
        im = b1 ? -h : h;
      }
      v[2 * m] = re;
      v[2 * m + 1] = im;
    }
  } else {
#pragma unroll
    for (int m = 0; m < 24; ++m) v[m] = 0;
  }
  SIO<P>::store(seg_ptr_w<P>(dst, L), seg_norm(dst, L), nitems, j, v);
}

// Gauge compression: thread per lexicographic site, all four directions.
__global__ void pack_gauge_kernel(LatDesc L, const double2* __restrict__ links, double2* g64, float4* gdf, void* g32,
                                  int rec32, void* g16, int rec16) {
  const int lex = blockIdx.x * blockDim.x + threadIdx.x;
  const int V = 2 * L.Vh;
  if (lex >= V) return;
  int x = lex % L.X, r = lex / L.X;
  int y = r % L.Y;
  r /= L.Y;
  int z = r % L.Z, t = r / L.Z;
  const int p = (x + y + z + t) & 1;
  const int i = lex >> 1;
  const int Vh = L.Vh;
  for (int mu = 0; mu < 4; ++mu) {
    const double2* u = links + ((size_t)lex * 4 + mu) * 9;
    double2 e[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) e[k] = u[k];
    const size_t blk = (size_t)(p * 4 + mu);
    if (g64) {
#pragma unroll
      for (int k = 0; k < 9; ++k) g64[(blk * 9 + k) * Vh + i] = e[k];
    }
    if (gdf) {  // double-float: hi = the nearest float, lo = the nearest float to the remainder
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const float rh = (float)e[k].x, ih = (float)e[k].y;
        gdf[(blk * 9 + k) * Vh + i] = make_float4(rh, (float)(e[k].x - (double)rh), ih, (float)(e[k].y - (double)ih));
      }
    }
    if (g32) {
      float4* g = (float4*)g32;
      if (rec32 == 12) {
        g[(blk * 3 + 0) * Vh + i] = make_float4(e[0].x, e[0].y, e[1].x, e[1].y);
        g[(blk * 3 + 1) * Vh + i] = make_float4(e[2].x, e[2].y, e[3].x, e[3].y);
        g[(blk * 3 + 2) * Vh + i] = make_float4(e[4].x, e[4].y, e[5].x, e[5].y);
      } else {
        float ta = (float)atan2(e[0].y, e[0].x), tc = (float)atan2(e[6].y, e[6].x);
        g[(blk * 2 + 0) * Vh + i] = make_float4(e[1].x, e[1].y, e[2].x, e[2].y);
        g[(blk * 2 + 1) * Vh + i] = make_float4(e[3].x, e[3].y, ta, tc);
      }
    }
    if (g16) {
      // offset-binary 16-bit fixed point: u = round(x * 32767) + 32768
      auto u16 = [](double x) -> unsigned {
        double y = x * 32767.0;
        y = y > 32767.0 ? 32767.0 : (y < -32767.0 ? -32767.0 : y);
        return (unsigned)(__double2int_rn(y) + 32768);
      };
      auto pair = [&](double a, double b) -> unsigned { return u16(a) | (u16(b) << 16); };
      if (rec16 == 12) {
        uint2* g = (uint2*)g16;
        for (int k = 0; k < 3; ++k)
          g[(blk * 3 + k) * Vh + i] = make_uint2(pair(e[2 * k].x, e[2 * k].y), pair(e[2 * k + 1].x, e[2 * k + 1].y));
      } else {
        uint4* g = (uint4*)g16;
        const double ipi = 1.0 / 3.14159265358979323846;
        g[blk * Vh + i] = make_uint4(pair(e[1].x, e[1].y), pair(e[2].x, e[2].y), pair(e[3].x, e[3].y),
                                     pair(atan2(e[0].y, e[0].x) * ipi, atan2(e[6].y, e[6].x) * ipi));
      }
    }
  }
}

}  // namespace

namespace dl {

#define DISPATCH_P(prec, CALL) \
  switch (prec) {              \
    case P64: { constexpr int PP = P64; CALL; } break; \
    case P32: { constexpr int PP = P32; CALL; } break; \
    case P16: { constexpr int PP = P16; CALL; } break; \
    case PBF: { constexpr int PP = PBF; CALL; } break; \
    case PDF: { constexpr int PP = PDF; CALL; } break; \
    default: return cudaErrorInvalidValue; \
  }

cudaError_t pack(const Batch& B, int prec, int parity, FieldRef dst, const void* natural, int dtype, cudaStream_t st) {
  long long items = (long long)B.lat[0].Vh << B.lat[0].lognpad;
  int g = (int)((items + 255) / 256);
  if (!g) return cudaSuccess;
  DL_COUNT();
  DISPATCH_P(prec, (pack_kernel<PP><<<g, 256, 0, st>>>(B, parity, dst, natural, dtype)));
  return cudaGetLastError();
}

cudaError_t unpack(const Batch& B, int prec, int parity, void* natural, FieldRef src, int dtype, cudaStream_t st) {
  long long items = (long long)B.lat[0].Vh << B.lat[0].lognpad;
  int g = (int)((items + 255) / 256);
  if (!g) return cudaSuccess;
  DL_COUNT();
  DISPATCH_P(prec, (unpack_kernel<PP><<<g, 256, 0, st>>>(B, parity, natural, src, dtype)));
  return cudaGetLastError();
}

cudaError_t noise_z4(const Batch& Bin, int prec, int parity, FieldRef dst, unsigned long long seed,
                     unsigned long long first, int quadrant, cudaStream_t st, Slices S) {
  Batch B = Bin;
  int g = blocks_for(B, 256);
  if (!g) return cudaSuccess;
  if (S.ns == 0) S = Slices{0, 1, 1 << 30};  // every slice
  DL_COUNT();
  DISPATCH_P(prec, (noise_kernel<PP><<<g, 256, 0, st>>>(B, parity, dst, seed, first, quadrant, S)));
  return cudaGetLastError();
}

cudaError_t pack_gauge(const LatDesc& L, const double* links_dev, void* g64, void* gdf, void* g32, int rec32, void* g16,
                       int rec16, cudaStream_t st) {
  int V = 2 * L.Vh;
  DL_COUNT();
  pack_gauge_kernel<<<(V + 127) / 128, 128, 0, st>>>(L, (const double2*)links_dev, (double2*)g64, (float4*)gdf, g32, rec32,
                                                     g16, rec16);
  return cudaGetLastError();
}

}  // namespace dl
