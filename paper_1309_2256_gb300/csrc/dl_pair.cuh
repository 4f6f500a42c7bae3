// Two right-hand sides per thread in packed FP32 arithmetic (the FP32 and 16-bit
// stencils).
//
// A thread owns the adjacent items j0 = 2 jp and j0 + 1 (two columns of one site)
// and keeps every real of its spinors as a float2 pair (value of column j0, value of
// column j0 + 1).  The arithmetic of the hop (spin projection, SU(3) product,
// reconstruction) is the same for both columns, so every instruction is a packed
// two-lane FP32 operation (add/mul/fma .f32x2, sm_100 and later): half the
// instructions of the one-column kernel for the same arithmetic.  Each lane rounds
// exactly like the scalar FP32 operation it replaces.
//
// Memory: chunk k of items j0 and j0 + 1 are adjacent 16-byte chunks (items are the
// innermost index of every field), read and written as one 32-byte access.  Fields
// are cudaMalloc'd and lattice segments start at even items, so these accesses are
// 32-byte aligned (the launcher checks the base pointers).
#pragma once

#include "dl_internal.cuh"

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }

// 32-byte global accesses (ld/st .v8, sm_100 and later)
__device__ __forceinline__ void ld256(const void* p, unsigned (&v)[8]) {
  asm volatile("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "l"(p));
}
__device__ __forceinline__ void st256(void* p, const unsigned (&v)[8]) {
  asm volatile("st.global.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "r"(v[0]), "r"(v[1]), "r"(v[2]),
               "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}

// Offset-binary 16-bit value u of a word half as the float 2^23 + u (one byte permute);
// subtracting 2^23 + 32768 gives the signed fixed-point integer q exactly.
__device__ __forceinline__ float u16lo_biased(unsigned w) { return __int_as_float((int)__byte_perm(w, 0x4B000000u, 0x7610)); }
__device__ __forceinline__ float u16hi_biased(unsigned w) { return __int_as_float((int)__byte_perm(w, 0x4B000000u, 0x7632)); }
#define DL_Q_BIAS 8421376.0f  // 2^23 + 32768

template <int P> struct PIO;

// FP32: chunk k of an item = (re, im) of complexes 2k and 2k + 1
template <> struct PIO<P32> {
  // v = the 24 reals of items j0, j0 + 1; w = (1, 1): FP32 storage has no scale
  __device__ static __forceinline__ void load(const void* b, const float*, long long st, long long j0, float2 v[24],
                                              float2& w) {
    const float4* p = (const float4*)b;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      unsigned a[8];
      ld256(p + k * st + j0, a);
#pragma unroll
      for (int q = 0; q < 4; ++q) v[4 * k + q] = make_float2(__uint_as_float(a[q]), __uint_as_float(a[4 + q]));
    }
    w = make_float2(1.f, 1.f);
  }
  // the values themselves (w applied): identical for FP32
  __device__ static __forceinline__ void load_values(const void* b, const float* nrm, long long st, long long j0,
                                                     float2 v[24]) {
    float2 w;
    load(b, nrm, st, j0, v, w);
  }
  // store columns j0 (if w0) and j0 + 1 (if w1)
  __device__ static __forceinline__ void store(void* b, float*, long long st, long long j0, const float2 v[24], bool w0,
                                               bool w1) {
    float4* p = (float4*)b;
    if (w0 && w1) {
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        unsigned a[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          a[q] = __float_as_uint(v[4 * k + q].x);
          a[4 + q] = __float_as_uint(v[4 * k + q].y);
        }
        st256(p + k * st + j0, a);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        if (w0) p[k * st + j0] = make_float4(v[4 * k].x, v[4 * k + 1].x, v[4 * k + 2].x, v[4 * k + 3].x);
        if (w1) p[k * st + j0 + 1] = make_float4(v[4 * k].y, v[4 * k + 1].y, v[4 * k + 2].y, v[4 * k + 3].y);
      }
    }
  }
};

// 16-bit: chunk k of an item = 8 offset-binary 16-bit values (re, im of complexes
// 4k .. 4k + 3), one float scale per item (value = q * scale / 32767)
template <> struct PIO<P16> {
  // v = the integers q of items j0, j0 + 1 (exact), w = their scale / 32767
  __device__ static __forceinline__ void load(const void* b, const float* nrm, long long st, long long j0, float2 v[24],
                                              float2& w) {
    const uint4* p = (const uint4*)b;
    const float2 nn = __ldg((const float2*)(nrm + j0));
    w = mul2(nn, dup2(1.0f / 32767.0f));
    const float2 bias = dup2(-DL_Q_BIAS);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      unsigned a[8];
      ld256(p + k * st + j0, a);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        v[8 * k + 2 * q] = add2(make_float2(u16lo_biased(a[q]), u16lo_biased(a[4 + q])), bias);
        v[8 * k + 2 * q + 1] = add2(make_float2(u16hi_biased(a[q]), u16hi_biased(a[4 + q])), bias);
      }
    }
  }
  // v = the biased values 2^23 + 32768 + q (one byte permute each, no subtraction), for
  // project_biased_pair; w as in load
  __device__ static __forceinline__ void load_biased(const void* b, const float* nrm, long long st, long long j0,
                                                     float2 v[24], float2& w) {
    const uint4* p = (const uint4*)b;
    const float2 nn = __ldg((const float2*)(nrm + j0));
    w = mul2(nn, dup2(1.0f / 32767.0f));
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      unsigned a[8];
      ld256(p + k * st + j0, a);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        v[8 * k + 2 * q] = make_float2(u16lo_biased(a[q]), u16lo_biased(a[4 + q]));
        v[8 * k + 2 * q + 1] = make_float2(u16hi_biased(a[q]), u16hi_biased(a[4 + q]));
      }
    }
  }
  __device__ static __forceinline__ void load_values(const void* b, const float* nrm, long long st, long long j0,
                                                     float2 v[24]) {
    float2 w;
    load(b, nrm, st, j0, v, w);
#pragma unroll
    for (int m = 0; m < 24; ++m) v[m] = mul2(v[m], w);
  }
  __device__ static __forceinline__ void store(void* b, float* nrm, long long st, long long j0, const float2 v[24], bool w0,
                                               bool w1) {
    uint4* p = (uint4*)b;
    float m0 = 0.f, m1 = 0.f;
#pragma unroll
    for (int q = 0; q < 24; ++q) {
      m0 = fmaxf(m0, fabsf(v[q].x));
      m1 = fmaxf(m1, fabsf(v[q].y));
    }
    const float2 sc = make_float2(m0 > 0.f ? 32767.0f / m0 : 0.f, m1 > 0.f ? 32767.0f / m1 : 0.f);
    const float2 bias = dup2(DL_Q_BIAS);
    unsigned a[12], c[12];  // the words of column j0 (a) and j0 + 1 (c)
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      // round(v * sc) + 2^23 + 32768: the low 16 mantissa bits are the offset-binary value
      const float2 re = fma2(v[2 * q], sc, bias), im = fma2(v[2 * q + 1], sc, bias);
      a[q] = __byte_perm(__float_as_uint(re.x), __float_as_uint(im.x), 0x5410);
      c[q] = __byte_perm(__float_as_uint(re.y), __float_as_uint(im.y), 0x5410);
    }
    if (w0 && w1) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const unsigned o[8] = {a[4 * k], a[4 * k + 1], a[4 * k + 2], a[4 * k + 3],
                               c[4 * k], c[4 * k + 1], c[4 * k + 2], c[4 * k + 3]};
        st256(p + k * st + j0, o);
      }
      *(float2*)(nrm + j0) = make_float2(m0, m1);
    } else {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        if (w0) p[k * st + j0] = make_uint4(a[4 * k], a[4 * k + 1], a[4 * k + 2], a[4 * k + 3]);
        if (w1) p[k * st + j0 + 1] = make_uint4(c[4 * k], c[4 * k + 1], c[4 * k + 2], c[4 * k + 3]);
      }
      if (w0) nrm[j0] = m0;
      if (w1) nrm[j0 + 1] = m1;
    }
  }
};

// Hop contribution along mu with projector (1 + s gamma_mu) for both columns:
//   acc += w (1 + s gamma_mu) U' v,   U' = U (forward hop) or U^dagger (backward hop),
// with the link entries staged as float4 (re, re, im, im) (one value for both lanes)
// and w the per-column scale of the neighbour (16-bit storage) or 1.  In the chiral
// basis (1 + s gamma_mu) maps the lower spins onto the upper ones through the block
// G_mu (G_k = -i sigma_k, G_t = 1):  h = v_up + s G v_dn, chi = U' h,
// acc_up += w chi, acc_dn += s w G^dagger chi.
//
// project_pair forms h for a run-time sign s; apply_pair does the rest.
template <int MU>
__device__ __forceinline__ void project_pair(const float2 v[24], float2 s2, float2 hr[2][3], float2 hi[2][3]) {
  const float2 ns2 = neg2(s2);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float2 u0r = v[2 * c], u0i = v[2 * c + 1], u1r = v[6 + 2 * c], u1i = v[7 + 2 * c];
    const float2 d2r = v[12 + 2 * c], d2i = v[13 + 2 * c], d3r = v[18 + 2 * c], d3i = v[19 + 2 * c];
    if (MU == 0) {         // (G d)_0 = -i d3, (G d)_1 = -i d2
      hr[0][c] = fma2(s2, d3i, u0r); hi[0][c] = fma2(ns2, d3r, u0i);
      hr[1][c] = fma2(s2, d2i, u1r); hi[1][c] = fma2(ns2, d2r, u1i);
    } else if (MU == 1) {  // (G d)_0 = -d3, (G d)_1 = d2
      hr[0][c] = fma2(ns2, d3r, u0r); hi[0][c] = fma2(ns2, d3i, u0i);
      hr[1][c] = fma2(s2, d2r, u1r); hi[1][c] = fma2(s2, d2i, u1i);
    } else if (MU == 2) {  // (G d)_0 = -i d2, (G d)_1 = i d3
      hr[0][c] = fma2(s2, d2i, u0r); hi[0][c] = fma2(ns2, d2r, u0i);
      hr[1][c] = fma2(ns2, d3i, u1r); hi[1][c] = fma2(s2, d3r, u1i);
    } else {               // G = 1
      hr[0][c] = fma2(s2, d2r, u0r); hi[0][c] = fma2(s2, d2i, u0i);
      hr[1][c] = fma2(s2, d3r, u1r); hi[1][c] = fma2(s2, d3i, u1i);
    }
  }
}

// The same projection on 16-bit offset-binary values held as B + q, B = 2^23 + 32768
// (PIO<P16>::load_biased), for a sign S known at compile time: every entry of h is an
// integer q_u + q_d or q_u - q_d.  A difference of two biased values is one exact
// subtraction (both lie in [2^23, 2^24)); a sum first takes 2B from one operand (q_u - B,
// an integer below 2^24 in magnitude, exact) and then adds the other (the exact sum is a
// small integer).  So h is bit-identical to project_pair on the decoded integers, with
// one or two instructions per entry instead of three.
template <int MU, int S>
__device__ __forceinline__ void project_biased_pair(const float2 v[24], float2 hr[2][3], float2 hi[2][3]) {
  const float2 m2b = dup2(-2.0f * DL_Q_BIAS), mone = dup2(-1.0f);
#define DL_PM(U, D, SIG) ((SIG) > 0 ? add2(add2((U), m2b), (D)) : fma2(mone, (D), (U)))
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float2 u0r = v[2 * c], u0i = v[2 * c + 1], u1r = v[6 + 2 * c], u1i = v[7 + 2 * c];
    const float2 d2r = v[12 + 2 * c], d2i = v[13 + 2 * c], d3r = v[18 + 2 * c], d3i = v[19 + 2 * c];
    if (MU == 0) {
      hr[0][c] = DL_PM(u0r, d3i, S); hi[0][c] = DL_PM(u0i, d3r, -S);
      hr[1][c] = DL_PM(u1r, d2i, S); hi[1][c] = DL_PM(u1i, d2r, -S);
    } else if (MU == 1) {
      hr[0][c] = DL_PM(u0r, d3r, -S); hi[0][c] = DL_PM(u0i, d3i, -S);
      hr[1][c] = DL_PM(u1r, d2r, S); hi[1][c] = DL_PM(u1i, d2i, S);
    } else if (MU == 2) {
      hr[0][c] = DL_PM(u0r, d2i, S); hi[0][c] = DL_PM(u0i, d2r, -S);
      hr[1][c] = DL_PM(u1r, d3i, -S); hi[1][c] = DL_PM(u1i, d3r, S);
    } else {
      hr[0][c] = DL_PM(u0r, d2r, S); hi[0][c] = DL_PM(u0i, d2i, S);
      hr[1][c] = DL_PM(u1r, d3r, S); hi[1][c] = DL_PM(u1i, d3i, S);
    }
  }
#undef DL_PM
}

template <int MU, bool BWD>
__device__ __forceinline__ void apply_pair(float2 acc[24], const float2 hr[2][3], const float2 hi[2][3],
                                           const float4* __restrict__ u, float2 s2, float2 w2) {
  // chi = U' h: (ur + i ui)(hr + i hi) = (ur hr - ui hi) + i (ur hi + ui hr); for
  // U^dagger the entry is conj(U_ba): ui changes sign
  float2 cr[2][3], ci[2][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float4 e = BWD ? u[3 * b + a] : u[3 * a + b];
      const float2 ur = make_float2(e.x, e.y), ui = make_float2(e.z, e.w);
#pragma unroll
      for (int sp = 0; sp < 2; ++sp) {
        const float2 pr = BWD ? hi[sp][b] : neg2(hi[sp][b]);  // multiplies ui in the real part
        const float2 pi = BWD ? neg2(hr[sp][b]) : hr[sp][b];  // multiplies ui in the imaginary part
        if (b == 0) {
          cr[sp][a] = fma2(ui, pr, mul2(ur, hr[sp][b]));
          ci[sp][a] = fma2(ui, pi, mul2(ur, hi[sp][b]));
        } else {
          cr[sp][a] = fma2(ui, pr, fma2(ur, hr[sp][b], cr[sp][a]));
          ci[sp][a] = fma2(ui, pi, fma2(ur, hi[sp][b], ci[sp][a]));
        }
      }
    }
  }
  const float2 sw = mul2(s2, w2), nsw = neg2(sw);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float2 c0r = cr[0][c], c0i = ci[0][c], c1r = cr[1][c], c1i = ci[1][c];
    acc[2 * c] = fma2(w2, c0r, acc[2 * c]);
    acc[2 * c + 1] = fma2(w2, c0i, acc[2 * c + 1]);
    acc[6 + 2 * c] = fma2(w2, c1r, acc[6 + 2 * c]);
    acc[7 + 2 * c] = fma2(w2, c1i, acc[7 + 2 * c]);
    float2 *a2r = &acc[12 + 2 * c], *a2i = &acc[13 + 2 * c], *a3r = &acc[18 + 2 * c], *a3i = &acc[19 + 2 * c];
    if (MU == 0) {         // G^+ chi = (i c1, i c0)
      *a2r = fma2(nsw, c1i, *a2r); *a2i = fma2(sw, c1r, *a2i);
      *a3r = fma2(nsw, c0i, *a3r); *a3i = fma2(sw, c0r, *a3i);
    } else if (MU == 1) {  // (c1, -c0)
      *a2r = fma2(sw, c1r, *a2r); *a2i = fma2(sw, c1i, *a2i);
      *a3r = fma2(nsw, c0r, *a3r); *a3i = fma2(nsw, c0i, *a3i);
    } else if (MU == 2) {  // (i c0, -i c1)
      *a2r = fma2(nsw, c0i, *a2r); *a2i = fma2(sw, c0r, *a2i);
      *a3r = fma2(sw, c1i, *a3r); *a3i = fma2(nsw, c1r, *a3i);
    } else {               // (c0, c1)
      *a2r = fma2(sw, c0r, *a2r); *a2i = fma2(sw, c0i, *a2i);
      *a3r = fma2(sw, c1r, *a3r); *a3i = fma2(sw, c1i, *a3i);
    }
  }
}

// (a + i b gamma_5) v for both columns, gamma_5 = diag(1, 1, -1, -1)
__device__ __forceinline__ void twist_pair(float2 v[24], float a, float b) {
  const float2 a2 = dup2(a);
#pragma unroll
  for (int m = 0; m < 12; ++m) {
    const float2 bb = dup2(m < 6 ? b : -b);
    const float2 re = v[2 * m], im = v[2 * m + 1];
    v[2 * m] = fma2(a2, re, mul2(neg2(bb), im));
    v[2 * m + 1] = fma2(a2, im, mul2(bb, re));
  }
}

// Per-column block reduction for two columns per thread (deterministic): thread t
// holds the values of columns 2 (t mod npad/2) and 2 (t mod npad/2) + 1 of its site;
// blockDim.x = 128.  Writes partial[col * pstride + blockIdx.x] for col < npad.
__device__ __forceinline__ void block_reduce_pairs(double v0, double v1, int npad, double* partial, int pstride) {
  __shared__ double sred[4][DL_MAXC];
  const int hp = npad >> 1;
  for (int off = 16; off >= hp; off >>= 1) {
    v0 += __shfl_xor_sync(0xffffffffu, v0, off);
    v1 += __shfl_xor_sync(0xffffffffu, v1, off);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane < hp) {
    sred[warp][2 * lane] = v0;
    sred[warp][2 * lane + 1] = v1;
  }
  __syncthreads();
  if (threadIdx.x < npad) {
    double s = 0.0;
    for (int w = 0; w < 4; ++w) s += sred[w][threadIdx.x];
    partial[(size_t)threadIdx.x * pstride + blockIdx.x] = s;
  }
}
