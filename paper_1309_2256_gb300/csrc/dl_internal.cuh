// Internal definitions shared by the discloop CUDA translation units.
//
// Device layouts (all 16-byte chunks so that every load/store is 128-bit):
//   spinor parity field, per lattice: chunk k of item j at  base + k*(Vh*npad) + j,
//     item j = site*npad + column, npad = 2^lognpad >= active columns.
//     F64: 12 chunks of double2 (one complex each, m = 3*spin + colour)
//     F32:  6 chunks of float4  (complex 2k, 2k+1)
//     16-bit: 3 chunks of uint4 (8 x 16 bit = complex 4k..4k+3) + float norm[item];
//           fixed point, value = q * norm / 32767 with norm the item's max |re|,|im|,
//           q stored offset-binary (q + 32768)
//   gauge field, per lattice: chunk k of link (parity p, mu, site i) at
//     base + ((p*4 + mu)*GK + k)*Vh + i
//     F64 recon 18: 9 double2 (row-major complex entries)
//     F32 recon 12: 3 float4  (rows 0 and 1), row 2 = conj(row0 x row1)
//     F32 recon  8: 2 float4  (a1, a2, b0, arg a0, arg c0)
//     16-bit recon 12: 3 uint2 (rows 0 and 1, int16 fixed point q / 32767)
//     16-bit recon  8: 1 uint4 (a1, a2, b0, arg a0 / pi, arg c0 / pi as int16 fixed point)
// Several lattices can share one launch ("batch"): lattice l owns blocks
// [blk_begin_l, blk_begin_{l+1}) and its own segment of every field.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "dl_df.cuh"
#include <stdint.h>

#include <string>
#include <type_traits>

#define DL_MAX_LAT 16
#define DL_MAXC 32  // max columns (right-hand sides) per lattice segment

// Storage formats: P64 FP64 (natural-format input/output), P32 FP32, P16 16-bit
// fixed point, PBF bfloat16 (network activations), PDF double-float (the
// high-precision arithmetic of the solver on GB300, see dl_df.cuh).
enum { P64 = 0, P32 = 1, P16 = 2, PBF = 3, PDF = 4 };

// ---------------------------------------------------------------- batch
struct LatDesc {
  int X, Y, Z, T;
  int Vh;            // sites per parity
  int lognpad;       // columns padded to 2^lognpad
  int ncol;          // active columns
  int rhs_base;      // global column index of column 0
  long long item_off;   // item offset of this lattice in a parity field
  long long gsite_off;  // parity-site offset of this lattice in the gauge arrays
  double tbc;        // time-boundary factor
  double kappa, amu;
  long long noise_base;  // noise index of column 0 (instances of one lattice differ)
};

struct Batch {
  int nlat;
  int pstride;  // column stride of the partial-sum buffer (>= blocks of any launch)
  int blk_begin[DL_MAX_LAT + 1];
  LatDesc lat[DL_MAX_LAT];
};

__device__ __forceinline__ int find_lat(const Batch& B, int blk) {
  int l = 0;
#pragma unroll 1
  for (int k = 1; k < B.nlat; ++k)
    if (blk >= B.blk_begin[k]) l = k;
  return l;
}

// Coordinates of checkerboard site i of parity p.
__device__ __forceinline__ void cb_coords(const LatDesc& L, int i, int p, int& x, int& y, int& z, int& t) {
  int full = 2 * i;
  int xh = full % L.X;
  int rest = full / L.X;
  y = rest % L.Y;
  rest /= L.Y;
  z = rest % L.Z;
  t = rest / L.Z;
  x = xh + ((y + z + t + p) & 1);
}

__device__ __forceinline__ int lex_of(const LatDesc& L, int x, int y, int z, int t) {
  return x + L.X * (y + L.Y * (z + L.Z * t));
}

// ---------------------------------------------------------------- spinor IO
template <int P> struct SIO;

template <> struct SIO<P64> {
  typedef double real;
  static constexpr int K = 12;
  __device__ static __forceinline__ void load(const void* b, const float*, long long st, long long j, double v[24]) {
    const double2* p = (const double2*)b;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      double2 c = __ldg(p + k * st + j);
      v[2 * k] = c.x;
      v[2 * k + 1] = c.y;
    }
  }
  __device__ static __forceinline__ void store(void* b, float*, long long st, long long j, const double v[24]) {
    double2* p = (double2*)b;
#pragma unroll
    for (int k = 0; k < 12; ++k) p[k * st + j] = make_double2(v[2 * k], v[2 * k + 1]);
  }
};

template <> struct SIO<P32> {
  typedef float real;
  static constexpr int K = 6;
  __device__ static __forceinline__ void load(const void* b, const float*, long long st, long long j, float v[24]) {
    const float4* p = (const float4*)b;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      float4 c = __ldg(p + k * st + j);
      v[4 * k] = c.x;
      v[4 * k + 1] = c.y;
      v[4 * k + 2] = c.z;
      v[4 * k + 3] = c.w;
    }
  }
  __device__ static __forceinline__ void store(void* b, float*, long long st, long long j, const float v[24]) {
    float4* p = (float4*)b;
#pragma unroll
    for (int k = 0; k < 6; ++k) p[k * st + j] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
  }
};

// 16-bit storage: 16-bit fixed point scaled by the item's max |re|,|im|
// (value = q * norm / 32767, q in [-32767, 32767]), i.e. 15 bits of precision
// relative to the site.  q is stored offset by 32768 (u = q + 32768) so that
// decoding is one byte permute into the mantissa of 2^23 + u followed by an
// exact subtraction, and encoding is one fused multiply-add whose result's low
// 16 mantissa bits are u (round to nearest even) followed by a byte permute.
__device__ __forceinline__ float u16lo_to_q(unsigned w) {
  return __int_as_float((int)__byte_perm(w, 0x4B000000u, 0x7610)) - 8421376.0f;  // (2^23 + u) - (2^23 + 32768)
}
__device__ __forceinline__ float u16hi_to_q(unsigned w) {
  return __int_as_float((int)__byte_perm(w, 0x4B000000u, 0x7632)) - 8421376.0f;
}
// pack round(a), round(b) (|a|,|b| <= 32767) as offset-binary 16-bit pair
__device__ __forceinline__ unsigned q_to_u16pair(float a, float b) {
  const unsigned ua = (unsigned)__float_as_int(a + 8421376.0f);
  const unsigned ub = (unsigned)__float_as_int(b + 8421376.0f);
  return __byte_perm(ua, ub, 0x5410);
}

template <> struct SIO<P16> {
  typedef float real;
  static constexpr int K = 3;
  __device__ static __forceinline__ void load(const void* b, const float* nrm, long long st, long long j, float v[24]) {
    const uint4* p = (const uint4*)b;
    const float s = __ldg(nrm + j) * (1.0f / 32767.0f);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 c = __ldg(p + k * st + j);
      const unsigned w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        v[8 * k + 2 * q] = u16lo_to_q(w[q]) * s;
        v[8 * k + 2 * q + 1] = u16hi_to_q(w[q]) * s;
      }
    }
  }
  __device__ static __forceinline__ void store(void* b, float* nrm, long long st, long long j, const float v[24]) {
    uint4* p = (uint4*)b;
    float m = 0.f;
#pragma unroll
    for (int q = 0; q < 24; ++q) m = fmaxf(m, fabsf(v[q]));
    const float sc = m > 0.f ? 32767.0f / m : 0.f;
    nrm[j] = m;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      unsigned w[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) w[q] = q_to_u16pair(v[8 * k + 2 * q] * sc, v[8 * k + 2 * q + 1] * sc);
      p[k * st + j] = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
};

// double-float: 12 chunks of (re.hi, re.lo, im.hi, im.lo), 192 bytes like FP64
template <> struct SIO<PDF> {
  typedef dfloat real;
  static constexpr int K = 12;
  __device__ static __forceinline__ void load(const void* b, const float*, long long st, long long j, dfloat v[24]) {
    const float4* p = (const float4*)b;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      float4 c = __ldg(p + k * st + j);
      v[2 * k] = dfloat(c.x, c.y);
      v[2 * k + 1] = dfloat(c.z, c.w);
    }
  }
  __device__ static __forceinline__ void store(void* b, float*, long long st, long long j, const dfloat v[24]) {
    float4* p = (float4*)b;
#pragma unroll
    for (int k = 0; k < 12; ++k) p[k * st + j] = make_float4(v[2 * k].hi, v[2 * k].lo, v[2 * k + 1].hi, v[2 * k + 1].lo);
  }
};

// Neighbour spinor of the stencil as values v and a common factor w with
// spinor = w v: the 16-bit format's per-site scale is applied once to the
// hop's result (folded into the accumulation) instead of to 24 inputs.
template <int P>
__device__ __forceinline__ void load_hop(const void* b, const float* nrm, long long st, long long j,
                                         typename SIO<P>::real v[24], typename SIO<P>::real& w) {
  SIO<P>::load(b, nrm, st, j, v);
  w = 1;
}
template <>
__device__ __forceinline__ void load_hop<P16>(const void* b, const float* nrm, long long st, long long j, float v[24],
                                              float& w) {
  const uint4* p = (const uint4*)b;
  w = __ldg(nrm + j) * (1.0f / 32767.0f);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    uint4 c = __ldg(p + k * st + j);
    const unsigned q4[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      v[8 * k + 2 * q] = u16lo_to_q(q4[q]);
      v[8 * k + 2 * q + 1] = u16hi_to_q(q4[q]);
    }
  }
}

// bfloat16 storage (network activations): 3 chunks of 8 bf16, no scale
template <> struct SIO<PBF> {
  typedef float real;
  static constexpr int K = 3;
  __device__ static __forceinline__ void load(const void* b, const float*, long long st, long long j, float v[24]) {
    const uint4* p = (const uint4*)b;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 c = __ldg(p + k * st + j);
      const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&c);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float2 f = __bfloat1622float2(h[q]);
        v[8 * k + 2 * q] = f.x;
        v[8 * k + 2 * q + 1] = f.y;
      }
    }
  }
  __device__ static __forceinline__ void store(void* b, float*, long long st, long long j, const float v[24]) {
    uint4* p = (uint4*)b;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 c;
      __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&c);
#pragma unroll
      for (int q = 0; q < 4; ++q) h[q] = __floats2bfloat162_rn(v[8 * k + 2 * q], v[8 * k + 2 * q + 1]);
      p[k * st + j] = c;
    }
  }
};

// A parity field of the whole batch: data pointer to chunk 0 of the first
// lattice; lattice l's segment starts at chunk K*item_off_l (norms at item_off_l).
struct FieldRef {
  void* data;
  float* norm;
};

template <int P>
__device__ __forceinline__ const void* seg_ptr(const FieldRef& f, const LatDesc& L) {
  constexpr int bytes = 16;
  return (const char*)f.data + (size_t)SIO<P>::K * bytes * (size_t)L.item_off;
}
template <int P>
__device__ __forceinline__ void* seg_ptr_w(const FieldRef& f, const LatDesc& L) {
  return (char*)f.data + (size_t)SIO<P>::K * 16 * (size_t)L.item_off;
}
__device__ __forceinline__ float* seg_norm(const FieldRef& f, const LatDesc& L) {
  return f.norm ? f.norm + L.item_off : nullptr;
}

// ---------------------------------------------------------------- gauge IO
enum { G64R18 = 0, G32R12 = 1, G32R8 = 2, G16R12 = 3, G16R8 = 4, GDF18 = 5 };

template <int G> struct GIO;

template <typename R>
__device__ __forceinline__ void recon12(R u[18]) {
  // row 2 = conj(row0 x row1)
  R a0r = u[0], a0i = u[1], a1r = u[2], a1i = u[3], a2r = u[4], a2i = u[5];
  R b0r = u[6], b0i = u[7], b1r = u[8], b1i = u[9], b2r = u[10], b2i = u[11];
  u[12] = (a1r * b2r - a1i * b2i) - (a2r * b1r - a2i * b1i);
  u[13] = -((a1r * b2i + a1i * b2r) - (a2r * b1i + a2i * b1r));
  u[14] = (a2r * b0r - a2i * b0i) - (a0r * b2r - a0i * b2i);
  u[15] = -((a2r * b0i + a2i * b0r) - (a0r * b2i + a0i * b2r));
  u[16] = (a0r * b1r - a0i * b1i) - (a1r * b0r - a1i * b0i);
  u[17] = -((a0r * b1i + a0i * b1r) - (a1r * b0i + a1i * b0r));
}

// Rebuild an SU(3) matrix from (a1, a2, b0, arg a0, arg c0) using unitarity
// (unit first row and column) and U^dagger = adj(U) for det U = 1.
__device__ __forceinline__ void recon8(float a1r, float a1i, float a2r, float a2i, float b0r, float b0i, float ta,
                                       float tc, float u[18]) {
  float n = a1r * a1r + a1i * a1i + a2r * a2r + a2i * a2i;
  float ma0 = sqrtf(fmaxf(0.f, 1.f - n));
  float sa, ca, sc, cc;
  sincosf(ta, &sa, &ca);
  sincosf(tc, &sc, &cc);
  float a0r = ma0 * ca, a0i = ma0 * sa;
  float mc0 = sqrtf(fmaxf(0.f, n - (b0r * b0r + b0i * b0i)));  // 1 - |a0|^2 - |b0|^2
  float c0r = mc0 * cc, c0i = mc0 * sc;
  float in = 1.f / n;
  // conj helpers: x* = (xr, -xi)
  // b1 = -(a0* a1 b0 + a2* c0*) / n
  float t1r = (a0r * a1r + a0i * a1i), t1i = (a0r * a1i - a0i * a1r);  // a0* a1
  float t2r = t1r * b0r - t1i * b0i, t2i = t1r * b0i + t1i * b0r;      // a0* a1 b0
  float t3r = a2r * c0r - a2i * c0i, t3i = -(a2r * c0i + a2i * c0r);   // a2* c0* = conj(a2 c0)
  float b1r = -(t2r + t3r) * in, b1i = -(t2i + t3i) * in;
  // b2 = (a1* c0* - a0* a2 b0) / n
  float s1r = a1r * c0r - a1i * c0i, s1i = -(a1r * c0i + a1i * c0r);  // conj(a1 c0)
  float s2r = (a0r * a2r + a0i * a2i), s2i = (a0r * a2i - a0i * a2r);  // a0* a2
  float s3r = s2r * b0r - s2i * b0i, s3i = s2r * b0i + s2i * b0r;
  float b2r = (s1r - s3r) * in, b2i = (s1i - s3i) * in;
  // c1 = (a2* b0* - a0* a1 c0) / n
  float q1r = a2r * b0r - a2i * b0i, q1i = -(a2r * b0i + a2i * b0r);  // conj(a2 b0)
  float q2r = t1r * c0r - t1i * c0i, q2i = t1r * c0i + t1i * c0r;      // a0* a1 c0
  float c1r = (q1r - q2r) * in, c1i = (q1i - q2i) * in;
  // c2 = -(a0* a2 c0 + a1* b0*) / n
  float w1r = s2r * c0r - s2i * c0i, w1i = s2r * c0i + s2i * c0r;      // a0* a2 c0
  float w2r = a1r * b0r - a1i * b0i, w2i = -(a1r * b0i + a1i * b0r);  // conj(a1 b0)
  float c2r = -(w1r + w2r) * in, c2i = -(w1i + w2i) * in;
  u[0] = a0r; u[1] = a0i; u[2] = a1r; u[3] = a1i; u[4] = a2r; u[5] = a2i;
  u[6] = b0r; u[7] = b0i; u[8] = b1r; u[9] = b1i; u[10] = b2r; u[11] = b2i;
  u[12] = c0r; u[13] = c0i; u[14] = c1r; u[15] = c1i; u[16] = c2r; u[17] = c2i;
}

template <> struct GIO<G64R18> {
  typedef double real;
  static constexpr int GK = 9;
  typedef double2 chunk;
  __device__ static __forceinline__ void load(const void* b, int Vh, int p, int mu, int i, double u[18]) {
    const double2* g = (const double2*)b + (size_t)((p * 4 + mu) * 9) * Vh + i;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      double2 c = __ldg(g + (size_t)k * Vh);
      u[2 * k] = c.x;
      u[2 * k + 1] = c.y;
    }
  }
};
template <> struct GIO<G32R12> {
  typedef float real;
  static constexpr int GK = 3;
  typedef float4 chunk;
  __device__ static __forceinline__ void load(const void* b, int Vh, int p, int mu, int i, float u[18]) {
    const float4* g = (const float4*)b + (size_t)((p * 4 + mu) * 3) * Vh + i;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float4 c = __ldg(g + (size_t)k * Vh);
      u[4 * k] = c.x; u[4 * k + 1] = c.y; u[4 * k + 2] = c.z; u[4 * k + 3] = c.w;
    }
    recon12(u);
  }
};
template <> struct GIO<G32R8> {
  typedef float real;
  static constexpr int GK = 2;
  typedef float4 chunk;
  __device__ static __forceinline__ void load(const void* b, int Vh, int p, int mu, int i, float u[18]) {
    const float4* g = (const float4*)b + (size_t)((p * 4 + mu) * 2) * Vh + i;
    float4 c0 = __ldg(g), c1 = __ldg(g + Vh);
    recon8(c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w, u);
  }
};
// double-float links, all 18 reals: 9 chunks of (re.hi, re.lo, im.hi, im.lo)
template <> struct GIO<GDF18> {
  typedef dfloat real;
  static constexpr int GK = 9;
  typedef float4 chunk;
  __device__ static __forceinline__ void load(const void* b, int Vh, int p, int mu, int i, dfloat u[18]) {
    const float4* g = (const float4*)b + (size_t)((p * 4 + mu) * 9) * Vh + i;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      float4 c = __ldg(g + (size_t)k * Vh);
      u[2 * k] = dfloat(c.x, c.y);
      u[2 * k + 1] = dfloat(c.z, c.w);
    }
  }
};
// 16-bit links: fixed point q / 32767 stored offset by 32768 like the spinors
// (entries of an SU(3) matrix lie in [-1, 1]; recon-8 angles are stored / pi).
template <> struct GIO<G16R12> {
  typedef float real;
  static constexpr int GK = 3;
  typedef uint2 chunk;
  __device__ static __forceinline__ void load(const void* b, int Vh, int p, int mu, int i, float u[18]) {
    const uint2* g = (const uint2*)b + (size_t)((p * 4 + mu) * 3) * Vh + i;
    const float s = 1.0f / 32767.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint2 c = __ldg(g + (size_t)k * Vh);
      u[4 * k] = u16lo_to_q(c.x) * s;
      u[4 * k + 1] = u16hi_to_q(c.x) * s;
      u[4 * k + 2] = u16lo_to_q(c.y) * s;
      u[4 * k + 3] = u16hi_to_q(c.y) * s;
    }
    recon12(u);
  }
};
template <> struct GIO<G16R8> {
  typedef float real;
  static constexpr int GK = 1;
  typedef uint4 chunk;
  __device__ static __forceinline__ void load(const void* b, int Vh, int p, int mu, int i, float u[18]) {
    const uint4* g = (const uint4*)b + (size_t)((p * 4 + mu)) * Vh + i;
    uint4 c = __ldg(g);
    const float s = 1.0f / 32767.0f, pi = 3.14159265358979f;
    recon8(u16lo_to_q(c.x) * s, u16hi_to_q(c.x) * s, u16lo_to_q(c.y) * s, u16hi_to_q(c.y) * s, u16lo_to_q(c.z) * s,
           u16hi_to_q(c.z) * s, u16lo_to_q(c.w) * s * pi, u16hi_to_q(c.w) * s * pi, u);
  }
};

template <int G>
__device__ __forceinline__ const void* gauge_seg(const void* base, const LatDesc& L) {
  return (const char*)base + (size_t)sizeof(typename GIO<G>::chunk) * GIO<G>::GK * 8 * (size_t)L.gsite_off;
}

// ---------------------------------------------------------------- spin algebra
// Hop contribution along mu with projector (1 + s gamma_mu), colour matrix u
// (adjoint if DAGU):  acc += w (1 + s gamma_mu) U psi.
// With G_mu the upper-right block of gamma_mu (G_k = -i sigma_k, G_t = 1):
//   h = psi_up + s G psi_dn,  chi = U h,  acc_up += chi,  acc_dn += s G^dagger chi.
// s x for a projector sign s = +-1, and w x for the hop's common factor w: a
// multiplication in FP32/FP64, a sign flip for double-float (whose storage has
// no scale, so w = +-1 there).
template <typename R> __device__ __forceinline__ R sgn_mul(R s, R x) { return s * x; }
template <> __device__ __forceinline__ dfloat sgn_mul<dfloat>(dfloat s, dfloat x) { return s.hi > 0.f ? x : -x; }

template <typename R, bool DAGU, int mu>
__device__ __forceinline__ void hop_term(R acc[24], const R v[24], const R u[18], R s, R w) {
  R h[12];  // [spin 0..1][colour][re,im]
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    R u0r = v[2 * c], u0i = v[2 * c + 1];            // spin 0
    R u1r = v[6 + 2 * c], u1i = v[6 + 2 * c + 1];    // spin 1
    R d2r = v[12 + 2 * c], d2i = v[12 + 2 * c + 1];  // spin 2
    R d3r = v[18 + 2 * c], d3i = v[18 + 2 * c + 1];  // spin 3
    R h0r, h0i, h1r, h1i;
    if (mu == 0) {        // G = [[0,-i],[-i,0]]: (G d)_0 = -i d3, (G d)_1 = -i d2
      h0r = u0r + sgn_mul(s, d3i); h0i = u0i - sgn_mul(s, d3r);
      h1r = u1r + sgn_mul(s, d2i); h1i = u1i - sgn_mul(s, d2r);
    } else if (mu == 1) { // G = [[0,-1],[1,0]]: (G d)_0 = -d3, (G d)_1 = d2
      h0r = u0r - sgn_mul(s, d3r); h0i = u0i - sgn_mul(s, d3i);
      h1r = u1r + sgn_mul(s, d2r); h1i = u1i + sgn_mul(s, d2i);
    } else if (mu == 2) { // G = diag(-i, i): (G d)_0 = -i d2, (G d)_1 = i d3
      h0r = u0r + sgn_mul(s, d2i); h0i = u0i - sgn_mul(s, d2r);
      h1r = u1r - sgn_mul(s, d3i); h1i = u1i + sgn_mul(s, d3r);
    } else {              // G = 1
      h0r = u0r + sgn_mul(s, d2r); h0i = u0i + sgn_mul(s, d2i);
      h1r = u1r + sgn_mul(s, d3r); h1i = u1i + sgn_mul(s, d3i);
    }
    h[2 * c] = h0r; h[2 * c + 1] = h0i;
    h[6 + 2 * c] = h1r; h[6 + 2 * c + 1] = h1i;
  }
  R chi[12];
#pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      R re = 0, im = 0;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        R ur, ui;
        if (DAGU) { ur = u[2 * (3 * b + a)]; ui = -u[2 * (3 * b + a) + 1]; }
        else { ur = u[2 * (3 * a + b)]; ui = u[2 * (3 * a + b) + 1]; }
        R hr = h[6 * sp + 2 * b], hi = h[6 * sp + 2 * b + 1];
        re += ur * hr - ui * hi;
        im += ur * hi + ui * hr;
      }
      chi[6 * sp + 2 * a] = re;
      chi[6 * sp + 2 * a + 1] = im;
    }
  }
  const R sw = sgn_mul(s, w);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    R c0r = chi[2 * c], c0i = chi[2 * c + 1], c1r = chi[6 + 2 * c], c1i = chi[6 + 2 * c + 1];
    acc[2 * c] += sgn_mul(w, c0r); acc[2 * c + 1] += sgn_mul(w, c0i);
    acc[6 + 2 * c] += sgn_mul(w, c1r); acc[6 + 2 * c + 1] += sgn_mul(w, c1i);
    R l2r, l2i, l3r, l3i;  // G^dagger chi
    if (mu == 0) {        // G^+ = [[0,i],[i,0]]: (G^+ c)_0 = i c1, (G^+ c)_1 = i c0
      l2r = -c1i; l2i = c1r; l3r = -c0i; l3i = c0r;
    } else if (mu == 1) { // G^+ = [[0,1],[-1,0]]: (G^+ c)_0 = c1, (G^+ c)_1 = -c0
      l2r = c1r; l2i = c1i; l3r = -c0r; l3i = -c0i;
    } else if (mu == 2) { // G^+ = diag(i, -i)
      l2r = -c0i; l2i = c0r; l3r = c1i; l3i = -c1r;
    } else {
      l2r = c0r; l2i = c0i; l3r = c1r; l3i = c1i;
    }
    acc[12 + 2 * c] += sgn_mul(sw, l2r); acc[12 + 2 * c + 1] += sgn_mul(sw, l2i);
    acc[18 + 2 * c] += sgn_mul(sw, l3r); acc[18 + 2 * c + 1] += sgn_mul(sw, l3i);
  }
}

// The same hop in double-float with lazy sums (dl_df.cuh): acc holds unnormalised
// (hi, lo) pairs during the eight hops and is normalised once before the epilogue.
// The projector sign s and the factor w are +-1 here (double-float storage has no
// scale; the boundary sign is folded into the staged link).
template <bool DAGU, int mu>
__device__ __forceinline__ void hop_term_df(dfloat acc[24], const dfloat v[24], const dfloat u[18], dfloat s, dfloat w) {
  const bool sp_ = s.hi > 0.f, wp = w.hi > 0.f;
  auto sg = [](bool pos, const dfloat& x) { return pos ? x : -x; };
  dfloat hr[2][3], hi[2][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const dfloat u0r = v[2 * c], u0i = v[2 * c + 1], u1r = v[6 + 2 * c], u1i = v[7 + 2 * c];
    const dfloat d2r = v[12 + 2 * c], d2i = v[13 + 2 * c], d3r = v[18 + 2 * c], d3i = v[19 + 2 * c];
    if (mu == 0) {         // (G d)_0 = -i d3, (G d)_1 = -i d2
      hr[0][c] = df_add_lazy(u0r, sg(sp_, d3i)); hi[0][c] = df_add_lazy(u0i, sg(!sp_, d3r));
      hr[1][c] = df_add_lazy(u1r, sg(sp_, d2i)); hi[1][c] = df_add_lazy(u1i, sg(!sp_, d2r));
    } else if (mu == 1) {  // (G d)_0 = -d3, (G d)_1 = d2
      hr[0][c] = df_add_lazy(u0r, sg(!sp_, d3r)); hi[0][c] = df_add_lazy(u0i, sg(!sp_, d3i));
      hr[1][c] = df_add_lazy(u1r, sg(sp_, d2r)); hi[1][c] = df_add_lazy(u1i, sg(sp_, d2i));
    } else if (mu == 2) {  // (G d)_0 = -i d2, (G d)_1 = i d3
      hr[0][c] = df_add_lazy(u0r, sg(sp_, d2i)); hi[0][c] = df_add_lazy(u0i, sg(!sp_, d2r));
      hr[1][c] = df_add_lazy(u1r, sg(!sp_, d3i)); hi[1][c] = df_add_lazy(u1i, sg(sp_, d3r));
    } else {               // G = 1
      hr[0][c] = df_add_lazy(u0r, sg(sp_, d2r)); hi[0][c] = df_add_lazy(u0i, sg(sp_, d2i));
      hr[1][c] = df_add_lazy(u1r, sg(sp_, d3r)); hi[1][c] = df_add_lazy(u1i, sg(sp_, d3i));
    }
  }
  const bool sw = sp_ == wp;  // sign of s w
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
      // chi = U' h for output colour a of spin sp; U' = U or U^dagger (conj(U_ba))
      dfloat cr, ci;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const dfloat ur = DAGU ? u[2 * (3 * b + a)] : u[2 * (3 * a + b)];
        const dfloat ui = DAGU ? -u[2 * (3 * b + a) + 1] : u[2 * (3 * a + b) + 1];
        if (b == 0) {
          cr = df_mul_lazy(ur, hr[sp][b]);
          ci = df_mul_lazy(ur, hi[sp][b]);
        } else {
          df_acc_mul(cr, ur, hr[sp][b]);
          df_acc_mul(ci, ur, hi[sp][b]);
        }
        df_acc_mul(cr, -ui, hi[sp][b]);
        df_acc_mul(ci, ui, hr[sp][b]);
      }
      cr = df_normalize(cr);
      ci = df_normalize(ci);
      // acc_up += w chi;  acc_dn += s w G^dagger chi
      df_acc(acc[6 * sp + 2 * a], sg(wp, cr));
      df_acc(acc[6 * sp + 2 * a + 1], sg(wp, ci));
      // G^dagger maps upper spin sp to lower spin: mu 0: (i c1, i c0); 1: (c1, -c0);
      // 2: (i c0, -i c1); 3: (c0, c1)   [lower spin 2 from c_1 or c_0, lower 3 likewise]
      int lo_sp;
      bool neg, imul;
      if (mu == 0) { lo_sp = sp == 1 ? 2 : 3; neg = false; imul = true; }
      else if (mu == 1) { lo_sp = sp == 1 ? 2 : 3; neg = sp == 0; imul = false; }
      else if (mu == 2) { lo_sp = sp == 0 ? 2 : 3; neg = sp == 1; imul = true; }
      else { lo_sp = sp == 0 ? 2 : 3; neg = false; imul = false; }
      const bool pos = (sw != neg);  // overall sign of the term
      dfloat* t = &acc[6 * lo_sp + 2 * a];
      if (imul) {  // +-i (cr + i ci) = +-(-ci + i cr)
        df_acc(t[0], sg(!pos, ci));
        df_acc(t[1], sg(pos, cr));
      } else {
        df_acc(t[0], sg(pos, cr));
        df_acc(t[1], sg(pos, ci));
      }
    }
  }
}

// The double-float hop with the direction and dagger as runtime values: the stencil
// loops over its eight hops without unrolling, so one copy of this (long) body serves
// all of them and the kernel's code fits the instruction cache (unrolled, the eight
// specialised bodies made instruction fetch the kernel's main stall).
// (G d)_sp = c_sp d_{src_sp} with c in {+-1, +-i}; (G^+ chi)_{2,3} likewise from chi_{0,1}.
__device__ __forceinline__ dfloat df_sel(bool neg, const dfloat& x) { return neg ? -x : x; }
// c z for c = (imag ? i : 1) * (neg ? -1 : 1):  (re, im) of the product
__device__ __forceinline__ void df_cmul_unit(bool imag, bool neg, const dfloat& zr, const dfloat& zi, dfloat& re,
                                             dfloat& im) {
  re = imag ? df_sel(!neg, zi) : df_sel(neg, zr);  // i z = (-zi, zr)
  im = imag ? df_sel(neg, zr) : df_sel(neg, zi);
}
__device__ __forceinline__ void hop_term_df_rt(dfloat acc[24], const dfloat v[24], const dfloat u[18], bool spos, bool wpos, int mu,
                               bool dagu) {
  // projection coefficients (G d)_sp = c d_src: mu 0: (-i d3, -i d2); 1: (-d3, d2); 2: (-i d2, i d3); 3: (d2, d3)
  const bool pim = (mu == 0 || mu == 2);
  const int src0 = (mu == 0 || mu == 1) ? 3 : 2, src1 = 5 - src0;
  const bool neg0 = mu != 3, neg1 = mu == 0;  // sign of c for sp = 0, 1 (before the projector sign s)
  dfloat hr[2][3], hi[2][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
      const bool from3 = (sp ? src1 : src0) == 3;  // selects, not a runtime index (keeps v in registers)
      const dfloat dr = from3 ? v[18 + 2 * c] : v[12 + 2 * c], di = from3 ? v[19 + 2 * c] : v[13 + 2 * c];
      const bool ng = (sp ? neg1 : neg0) != !spos;  // times the projector sign s
      dfloat gr, gi;
      df_cmul_unit(pim, ng, dr, di, gr, gi);
      hr[sp][c] = df_add_lazy(v[6 * sp + 2 * c], gr);
      hi[sp][c] = df_add_lazy(v[6 * sp + 2 * c + 1], gi);
    }
  }
  // G^+ chi: lower spin 2 from upper spin lsrc2 times c2, lower 3 from lsrc3 times c3:
  // mu 0: (i c1, i c0); 1: (c1, -c0); 2: (i c0, -i c1); 3: (c0, c1)
  const int lsrc2 = (mu == 0 || mu == 1) ? 1 : 0;
  const bool lneg2 = false, lneg3 = (mu == 1 || mu == 2);
  const bool sw = spos == wpos;  // sign of s w
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
      dfloat cr, ci;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const dfloat ur = dagu ? u[2 * (3 * b + a)] : u[2 * (3 * a + b)];
        const dfloat ui = dagu ? -u[2 * (3 * b + a) + 1] : u[2 * (3 * a + b) + 1];
        if (b == 0) {
          cr = df_mul_lazy(ur, hr[sp][b]);
          ci = df_mul_lazy(ur, hi[sp][b]);
        } else {
          df_acc_mul(cr, ur, hr[sp][b]);
          df_acc_mul(ci, ur, hi[sp][b]);
        }
        df_acc_mul(cr, -ui, hi[sp][b]);
        df_acc_mul(ci, ui, hr[sp][b]);
      }
      cr = df_normalize(cr);
      ci = df_normalize(ci);
      df_acc(acc[6 * sp + 2 * a], df_sel(!wpos, cr));
      df_acc(acc[6 * sp + 2 * a + 1], df_sel(!wpos, ci));
      const bool to2 = sp == lsrc2;  // lower spin 2 or 3 (a uniform branch, constant indices)
      const bool ln = (to2 ? lneg2 : lneg3) != !sw;
      dfloat tr, ti;
      df_cmul_unit(pim, ln, cr, ci, tr, ti);
      if (to2) {
        df_acc(acc[12 + 2 * a], tr);
        df_acc(acc[13 + 2 * a], ti);
      } else {
        df_acc(acc[18 + 2 * a], tr);
        df_acc(acc[19 + 2 * a], ti);
      }
    }
  }
}

// The hop of the staged and direct stencils for every arithmetic type.
template <typename R, bool DAGU, int mu>
__device__ __forceinline__ void hop_any(R acc[24], const R v[24], const R u[18], R s, R w) {
  if constexpr (std::is_same<R, dfloat>::value) hop_term_df<DAGU, mu>(acc, v, u, s, w);
  else hop_term<R, DAGU, mu>(acc, v, u, s, w);
}
// after the hops: lazy double-float sums become dfloats again
template <typename R>
__device__ __forceinline__ void hop_finish(R acc[24]) {
  if constexpr (std::is_same<R, dfloat>::value) {
#pragma unroll
    for (int m = 0; m < 24; ++m) acc[m] = df_normalize(acc[m]);
  }
}

// (a + i b gamma_5) v, gamma_5 = diag(1,1,-1,-1)
template <typename R>
__device__ __forceinline__ void twist_apply(R v[24], R a, R b) {
#pragma unroll
  for (int m = 0; m < 12; ++m) {
    R bb = (m < 6) ? b : -b;
    R re = v[2 * m], im = v[2 * m + 1];
    v[2 * m] = a * re - bb * im;
    v[2 * m + 1] = a * im + bb * re;
  }
}

// Per-column block reduction (deterministic).  Each thread contributes val for
// column col = (its item index) & (npad-1); blockDim.x is a multiple of 32 and
// npad <= 32.  Writes partial[col * pstride + blockIdx.x] for col < npad
// (column-major, so the final per-column sum reads contiguous memory).
__device__ __forceinline__ void block_reduce_cols(double val, int npad, double* partial, int pstride) {
  __shared__ double sred[32][DL_MAXC];
  for (int off = 16; off >= npad; off >>= 1) val += __shfl_xor_sync(0xffffffffu, val, off);
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane < npad) sred[warp][lane] = val;
  __syncthreads();
  if (threadIdx.x < npad) {
    double s = 0.0;
    int nw = blockDim.x >> 5;
    for (int w = 0; w < nw; ++w) s += sred[w][threadIdx.x];
    partial[(size_t)threadIdx.x * pstride + blockIdx.x] = s;
  }
}

// Time slices a contraction covers: t = t0 + k dt for k < ns (all T slices: 0, 1, T).
// Time-diluted sources (Sec. 2.3) are zero off their slices, so only those are contracted.
struct Slices {
  int t0, dt, ns;
};
__host__ __device__ __forceinline__ Slices all_slices(int T) { return Slices{0, 1, T}; }
// index k of slice t in the set, or -1
__host__ __device__ __forceinline__ int slice_index(const Slices& S, int t) {
  const int d = t - S.t0;
  if (d < 0 || d % S.dt != 0 || d / S.dt >= S.ns) return -1;
  return d / S.dt;
}

// ---------------------------------------------------------------- host side
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// Error plumbing: every launcher returns cudaError_t; the API layer maps it.
#define DL_CUDA_TRY(expr)                       \
  do {                                          \
    cudaError_t _e = (expr);                    \
    if (_e != cudaSuccess) return _e;           \
  } while (0)

// Epilogue parameters of a hop kernel for one lattice:
//   out = T1 (c * D^{(dag)} in + T2 aux),  T = a + i b gamma_5
struct Epi {
  double c, a1, b1, a2, b2;
  float cf, a1f, b1f, a2f, b2f;       // the same coefficients rounded once to FP32 (FP32 and 16-bit kernels)
  float cl, a1l, b1l, a2l, b2l;       // and the remainders: (xf, xl) is the double-float value
};
// An epilogue coefficient in the kernel's arithmetic type: GB300 issues FP64
// (and FP64<->FP32 conversion) instructions at a small fraction of the FP32
// rate, so the FP32 and double-float kernels read pre-split copies.
template <typename R> __device__ __forceinline__ R epc(double d, float f, float l);
template <> __device__ __forceinline__ double epc<double>(double d, float, float) { return d; }
template <> __device__ __forceinline__ float epc<float>(double, float f, float) { return f; }
template <> __device__ __forceinline__ dfloat epc<dfloat>(double, float f, float l) { return dfloat(f, l); }
struct EpiSet {
  Epi e[DL_MAX_LAT];
};

enum { EPI_PLAIN = 0, EPI_AUX = 1, EPI_AUX_NORM = 2, EPI_CG = 3 };

struct GaugeSet {
  const void* g64;
  const void* g32;
  const void* g16;
  const void* gdf;  // double-float copy of the FP64 links
};

// Every kernel launch is counted (host side) for the launch statistics of the C ABI.
void dl_count_launch();
#define DL_COUNT() dl_count_launch()

// Launchers (defined in the .cu files).
namespace dl {
int blocks_for(Batch& B, int threads);  // fills blk_begin, returns the grid size
cudaError_t dslash(const Batch& Bin, int prec, int grec, int epi, bool dag, int out_parity, FieldRef in, FieldRef aux,
                   FieldRef out, const GaugeSet& g, const EpiSet& ep, const int* active, double* partial,
                   FieldRef cg_r, FieldRef cg_y, FieldRef cg_p, const double* alpha, cudaStream_t st);

// Stencil launch statistics (process-wide) by class = (storage slot, epilogue, dagger):
// storage slot 0 double-float, 1 FP32, 2 16-bit, 3 IEEE FP64.  While enabled, every
// stencil launch outside stream capture is counted and timed with CUDA events (the
// graph body's launches are counted per replay by the solver: stencil_tally).
constexpr int DL_SCLASSES = 4 * 4 * 2;
struct StencilTally {
  long long n[DL_SCLASSES] = {0};
};
void stencil_prof_enable(bool on);    // resets the statistics
void stencil_prof_sampling(bool on);  // launches that are timed but not counted (extra profiling work)
void stencil_capture_begin();         // start tallying the launches captured on this thread
StencilTally stencil_capture_end();
void stencil_tally_add(const StencilTally& t, long long times);  // graph replays
// out[class][4] = (launches, timed launches, summed ms, summed site-column items of the timed ones)
cudaError_t stencil_prof_read(double* out);
}  // namespace dl
