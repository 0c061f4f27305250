// Shared-memory FFT building blocks for the circulant-embedded Toeplitz products
// (Sec. 3.1, Eq. be1: C = F^-1 diag(F c) F) and for the sine transforms.
//
// Convolutions only need  x (*) c = F^-1 (F x . F c): the forward transform here is a
// decimation-in-frequency FFT that leaves the spectrum in bit-reversed order, the
// inverse is the mirrored decimation-in-time FFT that takes bit-reversed input, and the
// kernel spectrum F c is stored in the same permuted order.  No reordering pass is ever
// needed.  Both transforms are unnormalised (the inverse returns n * x); the 1/n is
// folded into the stored kernel spectra.
//
// Twiddle tables: for every power of two n >= 2 up to the plan's maximum, the table of
// W_n^k = exp(-2 pi i k / n), k < n, sits at offset n-2 of one array.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ftoep {

// Float-float ("double-float") complex: each part is an unevaluated sum hi + lo of two
// floats (~48-bit significand), with error-free transformations (two-sum, FMA two-product)
// after Dekker and Knuth.  Used for the residual products of the mixed path, where about
// 1e-13 relative accuracy is needed and FP32 arithmetic is ~58x faster than FP64 on GB300.
struct FF {};
struct __align__(16) ff2 {
  float xh, xl, yh, yl;
};

template <typename T> struct VecOf;
template <> struct VecOf<double> { typedef double2 type; };
template <> struct VecOf<float> { typedef float2 type; };
template <> struct VecOf<FF> { typedef ff2 type; };

__device__ __forceinline__ void ff_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void ff_fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}
// (ah + al) + (bh + bl), accurate (both parts summed error-free)
__device__ __forceinline__ void ff_add(float ah, float al, float bh, float bl, float& rh, float& rl) {
  float s, e, t, f;
  ff_two_sum(ah, bh, s, e);
  ff_two_sum(al, bl, t, f);
  e += t;
  ff_fast_two_sum(s, e, s, e);
  e += f;
  ff_fast_two_sum(s, e, rh, rl);
}
// (ah + al) * (bh + bl)
__device__ __forceinline__ void ff_mul(float ah, float al, float bh, float bl, float& rh, float& rl) {
  const float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  ff_fast_two_sum(p, e, rh, rl);
}
// (ah + al) + (bh + bl) with one two-sum on the high parts: the error is bounded by a
// small multiple of 2^-48 (|a| + |b|) -- relative to the operands, not to the result.
// That is the bound the normwise rounding analysis of an FFT needs (every butterfly's
// error is charged against its inputs), and it costs 11 operations instead of 20.
__device__ __forceinline__ void ff_add_fast(float ah, float al, float bh, float bl, float& rh, float& rl) {
  float s, e;
  ff_two_sum(ah, bh, s, e);
  e += al + bl;
  ff_fast_two_sum(s, e, rh, rl);
}
__device__ __forceinline__ ff2 cadd(ff2 a, ff2 b) {
  ff2 r;
  ff_add_fast(a.xh, a.xl, b.xh, b.xl, r.xh, r.xl);
  ff_add_fast(a.yh, a.yl, b.yh, b.yl, r.yh, r.yl);
  return r;
}
__device__ __forceinline__ ff2 csub(ff2 a, ff2 b) {
  ff2 r;
  ff_add_fast(a.xh, a.xl, -b.xh, -b.xl, r.xh, r.xl);
  ff_add_fast(a.yh, a.yl, -b.yh, -b.yl, r.yh, r.yl);
  return r;
}
// p q - r s in float-float: the two high products exactly (FMA residuals), their
// difference by a two-sum, the cross terms of the low parts folded into the error word.
__device__ __forceinline__ void ff_dot2(float ph, float pl, float qh, float ql, float rh_, float rl_, float sh,
                                        float sl, float& oh, float& ol) {
  const float a = ph * qh, b = rh_ * sh;
  const float ea = fmaf(ph, qh, -a), eb = fmaf(rh_, sh, -b);
  float d, ed;
  ff_two_sum(a, -b, d, ed);
  float e = ed + (ea - eb);
  e = fmaf(ph, ql, e);
  e = fmaf(pl, qh, e);
  e = fmaf(-rh_, sl, e);
  e = fmaf(-rl_, sh, e);
  ff_fast_two_sum(d, e, oh, ol);
}
__device__ __forceinline__ ff2 cmul(ff2 a, ff2 b) {
  ff2 r;
  ff_dot2(a.xh, a.xl, b.xh, b.xl, a.yh, a.yl, b.yh, b.yl, r.xh, r.xl);    // ax bx - ay by
  ff_dot2(a.xh, a.xl, b.yh, b.yl, -a.yh, -a.yl, b.xh, b.xl, r.yh, r.yl);  // ax by + ay bx
  return r;
}
// a * conj(b)
__device__ __forceinline__ ff2 cmulc(ff2 a, ff2 b) {
  ff2 bc;
  bc.xh = b.xh;
  bc.xl = b.xl;
  bc.yh = -b.yh;
  bc.yl = -b.yl;
  return cmul(a, bc);
}
__device__ __forceinline__ ff2 mul_mi(ff2 a) {
  ff2 r;
  r.xh = a.yh;
  r.xl = a.yl;
  r.yh = -a.xh;
  r.yl = -a.xl;
  return r;
}
__device__ __forceinline__ ff2 mul_pi(ff2 a) {
  ff2 r;
  r.xh = -a.yh;
  r.xl = -a.yl;
  r.yh = a.xh;
  r.yl = a.xl;
  return r;
}
__device__ __forceinline__ ff2 ff2_from(double x, double y) {
  ff2 r;
  r.xh = (float)x;
  r.xl = (float)(x - (double)r.xh);
  r.yh = (float)y;
  r.yl = (float)(y - (double)r.yh);
  return r;
}

__device__ __forceinline__ double2 mkv(double x, double y) { return make_double2(x, y); }
__device__ __forceinline__ float2 mkv(float x, float y) { return make_float2(x, y); }

template <typename V> __device__ __forceinline__ V vzero() { V r; r.x = 0; r.y = 0; return r; }
template <> __device__ __forceinline__ ff2 vzero<ff2>() { ff2 r; r.xh = r.xl = r.yh = r.yl = 0.0f; return r; }
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { V r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { V r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
// a * b
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  V r;
  r.x = fma(a.x, b.x, -a.y * b.y);
  r.y = fma(a.x, b.y, a.y * b.x);
  return r;
}
// a * conj(b)
template <typename V> __device__ __forceinline__ V cmulc(V a, V b) {
  V r;
  r.x = fma(a.x, b.x, a.y * b.y);
  r.y = fma(a.y, b.x, -a.x * b.y);
  return r;
}
// a * (-i), a * (+i)
template <typename V> __device__ __forceinline__ V mul_mi(V a) { V r; r.x = a.y; r.y = -a.x; return r; }
template <typename V> __device__ __forceinline__ V mul_pi(V a) { V r; r.x = -a.y; r.y = a.x; return r; }

__device__ __forceinline__ int brev(int v, int logn) { return logn == 0 ? 0 : (int)(__brev((unsigned)v) >> (32 - logn)); }

// Forward (exponent -1) in-place radix-4/radix-2 DIF on `cnt` transforms of length
// n = 2^logn; transform t lives at a + t*ld.  Natural order in, bit-reversed order out.
// half_zero: the upper half of every input is zero and is not read.
// Called by all threads of the block; returns after a __syncthreads().
template <typename V>
__device__ void fft_dif(V* a, int logn, int cnt, int ld, const V* __restrict__ tw, bool half_zero) {
  if (logn == 0) return;
  const int n = 1 << logn;
  int gl = logn;  // log2 of the current group size
  bool first = true;
  if (logn & 1) {
    const V* w = tw + (n - 2);
    const int h = n >> 1;
    const int tot = cnt * h;
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
      const int t = e >> (logn - 1), i = e & (h - 1);
      V* b = a + (size_t)t * ld;
      const V u = b[i];
      if (half_zero) {
        b[i + h] = cmul(u, w[i]);
      } else {
        const V v = b[i + h];
        b[i] = cadd(u, v);
        b[i + h] = cmul(csub(u, v), w[i]);
      }
    }
    __syncthreads();
    gl = logn - 1;
    first = false;
  }
  const int quarter = n >> 2;
  for (; gl >= 2; gl -= 2) {
    const int g = 1 << gl, q = g >> 2;
    const V* w = tw + (g - 2);
    const bool hz = first && half_zero;
    const int tot = cnt * quarter;
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
      const int t = e >> (logn - 2), r = e & (quarter - 1);
      const int grp = r >> (gl - 2), i = r & (q - 1);
      V* b = a + (size_t)t * ld + grp * g + i;
      const V x0 = b[0], x1 = b[q];
      V x2, x3;
      if (hz) {
        x2 = vzero<V>();
        x3 = vzero<V>();
      } else {
        x2 = b[2 * q];
        x3 = b[3 * q];
      }
      const V s0 = cadd(x0, x2), s1 = cadd(x1, x3);
      const V d0 = csub(x0, x2), d1 = mul_mi(csub(x1, x3));
      b[0] = cadd(s0, s1);
      b[q] = cmul(csub(s0, s1), w[2 * i]);
      b[2 * q] = cmul(cadd(d0, d1), w[i]);
      b[3 * q] = cmul(csub(d0, d1), w[3 * i]);
    }
    __syncthreads();
    first = false;
  }
}

// Inverse (exponent +1, unnormalised) in-place DIT mirroring fft_dif: bit-reversed order
// in, natural order out.  keep: 0 = all outputs, 1 = only [n/2, n) is needed, 2 = only
// [0, n/2) is needed (the other half is left unspecified).
template <typename V>
__device__ void fft_dit(V* a, int logn, int cnt, int ld, const V* __restrict__ tw, int keep) {
  if (logn == 0) return;
  const int n = 1 << logn;
  const int top = logn - (logn & 1);
  const int quarter = n >> 2;
  for (int gl = 2; gl <= top; gl += 2) {
    const int g = 1 << gl, q = g >> 2;
    const V* w = tw + (g - 2);
    const bool last = (gl == logn);
    const int tot = cnt * quarter;
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
      const int t = e >> (logn - 2), r = e & (quarter - 1);
      const int grp = r >> (gl - 2), i = r & (q - 1);
      V* b = a + (size_t)t * ld + grp * g + i;
      const V z0 = b[0];
      const V t1 = cmulc(b[q], w[2 * i]);
      const V t2 = cmulc(b[2 * q], w[i]);
      const V t3 = cmulc(b[3 * q], w[3 * i]);
      const V y0 = cadd(z0, t1), y1 = csub(z0, t1);
      const V y2 = cadd(t2, t3), y3 = mul_pi(csub(t2, t3));
      if (!last || keep != 1) {
        b[0] = cadd(y0, y2);
        b[q] = cadd(y1, y3);
      }
      if (!last || keep != 2) {
        b[2 * q] = csub(y0, y2);
        b[3 * q] = csub(y1, y3);
      }
    }
    __syncthreads();
  }
  if (logn & 1) {
    const V* w = tw + (n - 2);
    const int h = n >> 1;
    const int tot = cnt * h;
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
      const int t = e >> (logn - 1), i = e & (h - 1);
      V* b = a + (size_t)t * ld;
      const V u = b[i];
      const V tt = cmulc(b[i + h], w[i]);
      if (keep != 2) b[i + h] = csub(u, tt);
      if (keep != 1) b[i] = cadd(u, tt);
    }
    __syncthreads();
  }
}

}  // namespace ftoep
