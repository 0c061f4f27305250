// Transform kernels: orthonormal sine transform (DST-I) along space, line packing,
// residual, reductions, kernel spectra and the circulant convolutions behind every
// Toeplitz product (Sec. 3.1, Eq. be1).
//
// Pair layout: the solver works on complex arrays z[P][ld] whose element (p, n) holds
// mode (or line) 2p in .x and 2p+1 in .y.  Convolution with a real kernel acts on the
// two components independently, so one complex FFT serves two real problems.
#include <cstdio>

#include "fft.cuh"
#include "fftr.cuh"
#include "internal.h"

namespace ftoep {

namespace {

constexpr int kThreads = 256;

template <typename T>
using Vt = typename VecOf<T>::type;

// Host-side copy of the pass radix of each arithmetic type (fftr.cuh EngineTraits).
template <typename T> struct EngineTraitsHost;
template <> struct EngineTraitsHost<float> { static constexpr int RB = 4; };
template <> struct EngineTraitsHost<double> { static constexpr int RB = 3; };
template <> struct EngineTraitsHost<FF> { static constexpr int RB = 3; };

inline void set_smem(const void* fn, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Conversions between double pairs and the storage types.
template <typename T> __device__ __forceinline__ typename VecOf<T>::type make_pair_of(double a, double b);
template <> __device__ __forceinline__ double2 make_pair_of<double>(double a, double b) { return make_double2(a, b); }
template <> __device__ __forceinline__ float2 make_pair_of<float>(double a, double b) { return make_float2((float)a, (float)b); }
template <> __device__ __forceinline__ ff2 make_pair_of<FF>(double a, double b) { return ff2_from(a, b); }
__device__ __forceinline__ double re_of(double2 v) { return v.x; }
__device__ __forceinline__ double im_of(double2 v) { return v.y; }
__device__ __forceinline__ double re_of(float2 v) { return (double)v.x; }
__device__ __forceinline__ double im_of(float2 v) { return (double)v.y; }
__device__ __forceinline__ double re_of(ff2 v) { return (double)v.xh + (double)v.xl; }
__device__ __forceinline__ double im_of(ff2 v) { return (double)v.yh + (double)v.yl; }

// ------------------------------------------------------------------ sine transform
//
// DST-I of length M via the odd extension y (length 2K, K = M+1): y_0 = y_K = 0,
// y_j = x_j, y_{2K-j} = -x_j.  Then FFT(y)_m = -2i sum_j x_j sin(pi j m / K).  Two real
// columns a (in .x) and b (in .y) share one complex FFT: FFT(a + i b)_m has real part
// 2 S_b[m] and imaginary part -2 S_a[m]; the orthonormal coefficient is
// sqrt(2/K) S[m] = (FFT value)/sqrt(2K).  The transform is its own inverse.

// Right-hand side at (j, n): f plus the initial-data terms.  Original form: wu0[n]*u0[j];
// difference form: -(S u0)_j with S the spatial operator (Dirichlet -u_xx or lambda).
__device__ __forceinline__ double rhs_value(const DstArgs& A, int64_t j, int64_t n) {
  double v = A.f[j * A.N + n];
  if (A.u0) {
    if (!A.diff_form) {
      v += A.wu0[n] * A.u0[j];
    } else if (A.space == 1) {
      const double um = j > 0 ? A.u0[j - 1] : 0.0;
      const double up = j + 1 < A.M ? A.u0[j + 1] : 0.0;
      v -= (2.0 * A.u0[j] - um - up) * A.inv_h2;
    } else {
      v -= A.lambda * A.u0[j];
    }
  }
  if (A.phi) v += A.wphi[n] * A.phi[j];
  return v;
}

constexpr int kDstThreads = 512;

template <typename T>
__global__ void __launch_bounds__(kDstThreads) dst_forward_kernel(DstArgs A, int C) {
  typedef Vt<T> V;
  V* z = (V*)A.z;
  const int64_t col0 = (int64_t)blockIdx.x * C;
  const int64_t M = A.M, N = A.N;
  const int64_t P = (M + 1) / 2;
  if (A.space == 0) {
    // no spatial transform: pairs of rows
    for (int64_t e = threadIdx.x; e < P * C; e += blockDim.x) {
      const int64_t p = e / C;
      const int c = (int)(e % C);
      const int64_t n = col0 + c;
      if (n >= A.ncols) continue;
      double v[2] = {0.0, 0.0};
      if (n < N) {
        for (int q = 0; q < 2; ++q) {
          const int64_t j = 2 * p + q;
          if (j >= M) continue;
          v[q] = rhs_value(A, j, n);
        }
      }
      const int64_t nout = (A.reverse && n < N) ? N - 1 - n : n;
      z[p * A.ld + nout] = mkv((T)v[0], (T)v[1]);
    }
    return;
  }
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int logK2 = A.logK2;
  const int K2 = 1 << logK2, K = K2 >> 1;
  const int lds = K2 + 1;
  const int CP = C >> 1;
  for (int cp = threadIdx.x; cp < CP; cp += blockDim.x) {
    sm[cp * lds] = vzero<V>();
    sm[cp * lds + K] = vzero<V>();
  }
  // four independent loads in flight per thread before the shared-memory stores
  const int64_t tot = M * C;
  for (int64_t e0 = threadIdx.x; e0 < tot; e0 += 4 * (int64_t)blockDim.x) {
    double v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t e = e0 + q * (int64_t)blockDim.x;
      const int64_t n = col0 + (e % C);
      v[q] = (e < tot && n < N) ? rhs_value(A, e / C, n) : 0.0;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t e = e0 + q * (int64_t)blockDim.x;
      if (e >= tot) break;
      const int c = (int)(e % C);
      const T tv = (T)v[q];
      V* col = sm + (c >> 1) * lds;
      const int pos = (int)(e / C) + 1;
      if (c & 1) {
        col[pos].y = tv;
        col[K2 - pos].y = -tv;
      } else {
        col[pos].x = tv;
        col[K2 - pos].x = -tv;
      }
    }
  }
  __syncthreads();
  fft_dif<V>(sm, logK2, CP, lds, (const V*)A.tw, false);
  const T scale = (T)(1.0 / sqrt(2.0 * (double)K));
  for (int64_t e = threadIdx.x; e < P * C; e += blockDim.x) {
    const int64_t p = e / C;
    const int c = (int)(e % C);
    const int64_t n = col0 + c;
    if (n >= A.ncols) continue;
    const V* col = sm + (c >> 1) * lds;
    const int m1 = (int)(2 * p + 1), m2 = m1 + 1;
    const V y1 = col[brev(m1, logK2)];
    const T v1 = (c & 1) ? y1.x : -y1.y;
    T v2 = (T)0;
    if (m2 <= M) {
      const V y2 = col[brev(m2, logK2)];
      v2 = (c & 1) ? y2.x : -y2.y;
    }
    const int64_t nout = (A.reverse && n < N) ? N - 1 - n : n;
    z[p * A.ld + nout] = mkv(v1 * scale, v2 * scale);
  }
}

template <typename T>
__global__ void __launch_bounds__(kDstThreads) dst_inverse_kernel(DstArgs A, int C) {
  typedef Vt<T> V;
  const V* z = (const V*)A.z;
  const int64_t col0 = (int64_t)blockIdx.x * C;
  const int64_t M = A.M, N = A.N;
  const int64_t P = (M + 1) / 2;
  if (A.space == 0) {
    for (int64_t e = threadIdx.x; e < P * C; e += blockDim.x) {
      const int64_t p = e / C;
      const int c = (int)(e % C);
      const int64_t n = col0 + c;
      if (n >= N) continue;
      const int64_t nin = A.reverse ? N - 1 - n : n;
      const V zz = z[p * A.ld + nin];
      for (int q = 0; q < 2; ++q) {
        const int64_t j = 2 * p + q;
        if (j >= M) continue;
        const double v = (double)(q ? zz.y : zz.x);
        double* dst = A.u + j * N + n;
        *dst = A.accumulate ? *dst + v : v;
      }
    }
    return;
  }
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int logK2 = A.logK2;
  const int K2 = 1 << logK2, K = K2 >> 1;
  const int lds = K2 + 1;
  const int CP = C >> 1;
  for (int cp = threadIdx.x; cp < CP; cp += blockDim.x) {
    sm[cp * lds] = vzero<V>();
    sm[cp * lds + K] = vzero<V>();
  }
  const int64_t tot = P * C;
  for (int64_t e0 = threadIdx.x; e0 < tot; e0 += 4 * (int64_t)blockDim.x) {
    V zq[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t e = e0 + q * (int64_t)blockDim.x;
      if (e < tot) {
        const int64_t n = col0 + (e % C);
        const int64_t nin = (A.reverse && n < N) ? N - 1 - n : n;
        zq[q] = z[(e / C) * A.ld + nin];
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t e = e0 + q * (int64_t)blockDim.x;
      if (e >= tot) break;
      const int64_t p = e / C;
      const int c = (int)(e % C);
      const V zz = zq[q];
      V* col = sm + (c >> 1) * lds;
      const int m1 = (int)(2 * p + 1), m2 = m1 + 1;
      if (c & 1) {
        col[m1].y = zz.x;
        col[K2 - m1].y = -zz.x;
        if (m2 <= M) {
          col[m2].y = zz.y;
          col[K2 - m2].y = -zz.y;
        }
      } else {
        col[m1].x = zz.x;
        col[K2 - m1].x = -zz.x;
        if (m2 <= M) {
          col[m2].x = zz.y;
          col[K2 - m2].x = -zz.y;
        }
      }
    }
  }
  __syncthreads();
  fft_dif<V>(sm, logK2, CP, lds, (const V*)A.tw, false);
  const double scale = 1.0 / sqrt(2.0 * (double)K);
  for (int64_t e = threadIdx.x; e < M * C; e += blockDim.x) {
    const int64_t j = e / C;
    const int c = (int)(e % C);
    const int64_t n = col0 + c;
    if (n >= N) continue;
    const V y = sm[(c >> 1) * lds + brev((int)j + 1, logK2)];
    const double v = (double)((c & 1) ? y.x : -y.y) * scale;
    double* dst = A.u + j * N + n;
    *dst = A.accumulate ? *dst + v : v;
  }
}

// Sine transform for any K = M+1 (Bluestein / chirp-z).  With W = exp(-2 pi i / L),
// L = 2K, and c_n = W^{n^2/2}: DFT(y)_k = c_k sum_n (y_n c_n) conj(c_{k-n}), a linear
// convolution that a cyclic one of length P >= 2L-1 reproduces exactly.  One block
// handles C time columns (C/2 complex column pairs, one P-buffer each).
template <typename T>
__global__ void __launch_bounds__(kDstThreads) dst_bluestein_kernel(DstArgs A, int C, int fwd) {
  typedef Vt<T> V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int64_t col0 = (int64_t)blockIdx.x * C;
  const int64_t M = A.M, N = A.N;
  const int64_t P2 = (M + 1) / 2;
  const int K = A.K, L = 2 * K;
  const int P = 1 << A.logP, H = P >> 1;
  const int lds = P + 1;
  const int CP = C >> 1;
  const V* chirp = (const V*)A.chirp;
  for (int e = threadIdx.x; e < CP * H; e += blockDim.x) sm[(e / H) * lds + (e % H)] = vzero<V>();
  __syncthreads();
  if (fwd) {
    const int64_t tot = M * C;
    for (int64_t e0 = threadIdx.x; e0 < tot; e0 += 4 * (int64_t)blockDim.x) {
      double vq[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t e = e0 + q * (int64_t)blockDim.x;
        const int64_t n = col0 + (e % C);
        vq[q] = (e < tot && n < N) ? rhs_value(A, e / C, n) : 0.0;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t e = e0 + q * (int64_t)blockDim.x;
        if (e >= tot) break;
        const int c = (int)(e % C);
        const T tv = (T)vq[q];
        V* col = sm + (c >> 1) * lds;
        const int pos = (int)(e / C) + 1;
        if (c & 1) {
          col[pos].y = tv;
          col[L - pos].y = -tv;
        } else {
          col[pos].x = tv;
          col[L - pos].x = -tv;
        }
      }
    }
  } else {
    const V* z = (const V*)A.z;
    const int64_t tot = P2 * C;
    for (int64_t e0 = threadIdx.x; e0 < tot; e0 += 4 * (int64_t)blockDim.x) {
     V zq[4];
#pragma unroll
     for (int q = 0; q < 4; ++q) {
      const int64_t e = e0 + q * (int64_t)blockDim.x;
      if (e < tot) {
        const int64_t n = col0 + (e % C);
        const int64_t nin = (A.reverse && n < N) ? N - 1 - n : n;
        zq[q] = z[(e / C) * A.ld + nin];
      }
     }
#pragma unroll
     for (int q = 0; q < 4; ++q) {
      const int64_t e = e0 + q * (int64_t)blockDim.x;
      if (e >= tot) break;
      const int64_t p = e / C;
      const int c = (int)(e % C);
      const V zz = zq[q];
      V* col = sm + (c >> 1) * lds;
      const int m1 = (int)(2 * p + 1), m2 = m1 + 1;
      if (c & 1) {
        col[m1].y = zz.x;
        col[L - m1].y = -zz.x;
        if (m2 <= M) {
          col[m2].y = zz.y;
          col[L - m2].y = -zz.y;
        }
      } else {
        col[m1].x = zz.x;
        col[L - m1].x = -zz.x;
        if (m2 <= M) {
          col[m2].x = zz.y;
          col[L - m2].x = -zz.y;
        }
      }
     }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < CP * L; e += blockDim.x) {
    V* q = sm + (e / L) * lds + (e % L);
    *q = cmul(*q, chirp[e % L]);
  }
  __syncthreads();
  const V* tw = (const V*)A.tw;
  fft_dif<V>(sm, A.logP, CP, lds, tw, true);
  const V* bs = (const V*)A.bspec;
  for (int e = threadIdx.x; e < CP * P; e += blockDim.x) {
    V* q = sm + (e / P) * lds + (e % P);
    *q = cmul(*q, bs[e % P]);
  }
  __syncthreads();
  fft_dit<V>(sm, A.logP, CP, lds, tw, 2);
  const double scale = 1.0 / sqrt(2.0 * (double)K);
  if (fwd) {
    V* z = (V*)A.z;
    for (int64_t e = threadIdx.x; e < P2 * C; e += blockDim.x) {
      const int64_t p = e / C;
      const int c = (int)(e % C);
      const int64_t n = col0 + c;
      if (n >= A.ncols) continue;
      const V* col = sm + (c >> 1) * lds;
      const int m1 = (int)(2 * p + 1), m2 = m1 + 1;
      const V y1 = cmul(col[m1], chirp[m1]);
      const T v1 = (c & 1) ? y1.x : -y1.y;
      T v2 = (T)0;
      if (m2 <= M) {
        const V y2 = cmul(col[m2], chirp[m2]);
        v2 = (c & 1) ? y2.x : -y2.y;
      }
      const int64_t nout = (A.reverse && n < N) ? N - 1 - n : n;
      z[p * A.ld + nout] = mkv((T)(v1 * (T)scale), (T)(v2 * (T)scale));
    }
  } else {
    for (int64_t e = threadIdx.x; e < M * C; e += blockDim.x) {
      const int64_t j = e / C;
      const int c = (int)(e % C);
      const int64_t n = col0 + c;
      if (n >= N) continue;
      const V y = cmul(sm[(c >> 1) * lds + (int)j + 1], chirp[j + 1]);
      const double v = (double)((c & 1) ? y.x : -y.y) * scale;
      double* dst = A.u + j * N + n;
      *dst = A.accumulate ? *dst + v : v;
    }
  }
}

template <typename T>
int bluestein_cols(int logP) {
  const size_t per_pair = ((size_t)(1 << logP) + 1) * sizeof(Vt<T>);
  int C = 4;
  while (C > 2 && (size_t)(C / 2) * per_pair > 160 * 1024) C >>= 1;
  return C;
}

template <typename T>
int dst_cols(int logK2) {
  // columns per block: as many as fit (even, <= 8) in ~160 KB of shared memory
  const size_t per_pair = ((size_t)(1 << logK2) + 1) * sizeof(Vt<T>);
  int C = 8;
  while (C > 2 && (size_t)(C / 2) * per_pair > 160 * 1024) C >>= 1;
  return C;
}

template <typename T>
void dst_launch(const DstArgs& a, bool fwd, cudaStream_t st) {
  if (a.space && a.bluestein) {
    const int C = bluestein_cols<T>(a.logP);
    const size_t smem = (size_t)(C / 2) * ((size_t)(1 << a.logP) + 1) * sizeof(Vt<T>);
    set_smem((const void*)dst_bluestein_kernel<T>, smem);
    dst_bluestein_kernel<T><<<(unsigned)((a.ncols + C - 1) / C), kDstThreads, smem, st>>>(a, C, fwd ? 1 : 0);
    return;
  }
  int C = a.space ? dst_cols<T>(a.logK2) : 8;
  size_t smem = a.space ? (size_t)(C / 2) * ((size_t)(1 << a.logK2) + 1) * sizeof(Vt<T>) : 0;
  dim3 grid((unsigned)((a.ncols + C - 1) / C));
  if (fwd) {
    set_smem((const void*)dst_forward_kernel<T>, smem);
    dst_forward_kernel<T><<<grid, kDstThreads, smem, st>>>(a, C);
  } else {
    set_smem((const void*)dst_inverse_kernel<T>, smem);
    dst_inverse_kernel<T><<<grid, kDstThreads, smem, st>>>(a, C);
  }
}

// ------------------------------------------------------------------ pack / unpack

template <typename T>
__global__ void pack_kernel(PackArgs A) {
  typedef Vt<T> V;
  const int64_t p = blockIdx.y;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= A.ld) return;
  double v0 = 0.0, v1 = 0.0;
  if (k < A.N) {
    const int64_t src = A.reverse ? A.N - 1 - k : k;
    v0 = A.x[(2 * p) * A.N + src];
    if (2 * p + 1 < A.nlines) v1 = A.x[(2 * p + 1) * A.N + src];
  }
  ((V*)A.z)[p * A.ld + k] = make_pair_of<T>(v0, v1);
}

template <typename T>
__global__ void unpack_kernel(PackArgs A) {
  typedef Vt<T> V;
  const int64_t p = blockIdx.y;
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= A.N) return;
  const int64_t k = A.reverse ? A.N - 1 - n : n;
  const V v = ((const V*)A.z)[p * A.ld + k];
  double* y0 = A.y + (2 * p) * A.N + n;
  *y0 = A.mode ? *y0 + re_of(v) : re_of(v);
  if (2 * p + 1 < A.nlines) {
    double* y1 = A.y + (2 * p + 1) * A.N + n;
    *y1 = A.mode ? *y1 + im_of(v) : im_of(v);
  }
}

// ------------------------------------------------------------------ time prefix sums

// One block per line; chunks of 4*kThreads elements, each thread a run of 4, block-wide
// exclusive scan of the run totals, carry between chunks.  Double precision throughout.
__global__ void __launch_bounds__(kThreads) scan_kernel(ScanArgs A) {
  __shared__ double wsum[kThreads / 32];
  __shared__ double carry_s;
  const int64_t j = blockIdx.x;
  const double* in = A.in + j * A.N;
  double* out = A.out + j * A.N;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t chunk = 4 * kThreads;
  double carry = 0.0;
  const int64_t nchunks = (A.N + chunk - 1) / chunk;
  for (int64_t ci = 0; ci < nchunks; ++ci) {
    // forward: chunks left to right, runs in order; reverse: mirror both
    const int64_t c0 = A.reverse ? A.N - (ci + 1) * chunk : ci * chunk;
    double v[4];
    double run = 0.0;
    for (int q = 0; q < 4; ++q) {
      const int64_t pos = A.reverse ? c0 + (chunk - 1 - (4 * threadIdx.x + q)) : c0 + 4 * threadIdx.x + q;
      v[q] = (pos >= 0 && pos < A.N) ? in[pos] : 0.0;
      run += v[q];
      v[q] = run;  // inclusive within the run
    }
    // exclusive scan of run totals across the block
    double x = run;
    for (int o = 1; o < 32; o <<= 1) {
      const double y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      double w = lane < kThreads / 32 ? wsum[lane] : 0.0;
      for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      if (lane < kThreads / 32) wsum[lane] = w;
      if (lane == kThreads / 32 - 1) carry_s = w;
    }
    __syncthreads();
    const double before = carry + (x - run) + (warp > 0 ? wsum[warp - 1] : 0.0);
    for (int q = 0; q < 4; ++q) {
      const int64_t pos = A.reverse ? c0 + (chunk - 1 - (4 * threadIdx.x + q)) : c0 + 4 * threadIdx.x + q;
      if (pos < 0 || pos >= A.N) continue;
      const double sum = A.tau * (before + v[q]);
      if (A.reverse) {
        out[pos] = sum;
      } else {
        const double base = A.accumulate ? out[pos] : (A.u0 ? A.u0[j] : 0.0);
        out[pos] = base + sum;
      }
    }
    carry += carry_s;
    __syncthreads();
  }
}

// ------------------------------------------------------------------ residual, dot

__global__ void residual_kernel(ResidualArgs A) {
  const int64_t j = blockIdx.y;
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= A.N) return;
  const int64_t idx = j * A.N + n;
  double v = A.f[idx];
  if (A.u0) v += A.wu0[n] * A.u0[j];
  if (A.phi) v += A.wphi[n] * A.phi[j];
  double tv;
  if (A.tu_ff) {
    const ff2 t = ((const ff2*)A.tu)[(j >> 1) * A.ld + n];
    tv = (j & 1) ? im_of(t) : re_of(t);
  } else {
    const double2 t = ((const double2*)A.tu)[(j >> 1) * A.ld + n];
    tv = (j & 1) ? t.y : t.x;
  }
  const double uj = A.u[idx];
  double s;
  if (A.space == 1) {
    const double um = j > 0 ? A.u[idx - A.N] : 0.0;
    const double up = j + 1 < A.M ? A.u[idx + A.N] : 0.0;
    s = (2.0 * uj - um - up) * A.inv_h2;
  } else {
    s = A.lambda * uj;
  }
  A.r[idx] = v - tv - s;
}

__global__ void dot_kernel(DotArgs A) {
  __shared__ double red[kThreads / 32];
  double acc = 0.0;
  const int64_t total = A.nlines * A.N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t l = e / A.N, n = e % A.N;
    const double2 t = A.tu[(l >> 1) * A.ld + n];
    acc += A.x[e] * ((l & 1) ? t.y : t.x);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    A.partial[blockIdx.x] = s;
  }
}

__global__ void sum_kernel(const double* partial, int n, double* out) {
  __shared__ double red[kThreads / 32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partial[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    *out = s;
  }
}

// ------------------------------------------------------------------ four-step split

struct Split {
  int logn, logn1, logn2;
};
inline Split split_of(int logn) { return Split{logn, logn / 2, logn - logn / 2}; }

template <typename T>
int four_step_cols(int logn1) {
  const size_t per = ((size_t)(1 << logn1) + 1) * sizeof(Vt<T>);
  int C = 8;
  while (C > 1 && (size_t)C * per > 160 * 1024) C >>= 1;
  return C;
}

// ------------------------------------------------------------------ spectra

template <typename TS>
__global__ void __launch_bounds__(kThreads) spec_smem_kernel(SpecArgs A) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double2* sm = reinterpret_cast<double2*>(smraw);
  const int n = 1 << A.logn;
  for (int k = threadIdx.x; k < n; k += blockDim.x) sm[k] = make_double2((k >= A.lo && k < A.hi) ? A.a[k] : 0.0, 0.0);
  __syncthreads();
  fft_dif<double2>(sm, A.logn, 1, 0, A.tw64, false);
  const double inv = 1.0 / (double)n;
  typedef Vt<TS> V;
  for (int k = threadIdx.x; k < n; k += blockDim.x) ((V*)A.out)[k] = make_pair_of<TS>(sm[k].x * inv, sm[k].y * inv);
}

__global__ void __launch_bounds__(kThreads) spec_col_kernel(SpecArgs A, int logn1, int logn2, int C) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double2* sm = reinterpret_cast<double2*>(smraw);
  const int n1 = 1 << logn1, n2 = 1 << logn2, n = n1 * n2;
  const int lds = n1 + 1;
  const int c0 = blockIdx.x * C;
  for (int e = threadIdx.x; e < n1 * C; e += blockDim.x) {
    const int j1 = e / C, c = e % C;
    const int64_t k = (int64_t)j1 * n2 + c0 + c;
    sm[c * lds + j1] = make_double2((k >= A.lo && k < A.hi) ? A.a[k] : 0.0, 0.0);
  }
  __syncthreads();
  fft_dif<double2>(sm, logn1, C, lds, A.tw64, false);
  const double2* twn = A.tw64 + (n - 2);
  for (int e = threadIdx.x; e < n1 * C; e += blockDim.x) {
    const int r = e / C, c = e % C;
    const int j2 = c0 + c;
    const int k1 = brev(r, logn1);
    A.scratch64[(int64_t)r * n2 + j2] = cmul(sm[c * lds + r], twn[(int64_t)j2 * k1 & (n - 1)]);
  }
}

template <typename TS>
__global__ void __launch_bounds__(kThreads) spec_row_kernel(SpecArgs A, int logn1, int logn2) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double2* sm = reinterpret_cast<double2*>(smraw);
  const int n2 = 1 << logn2;
  const int64_t n = (int64_t)n2 << logn1;
  const int r = blockIdx.x;
  for (int k = threadIdx.x; k < n2; k += blockDim.x) sm[k] = A.scratch64[(int64_t)r * n2 + k];
  __syncthreads();
  fft_dif<double2>(sm, logn2, 1, 0, A.tw64, false);
  const double inv = 1.0 / (double)n;
  typedef Vt<TS> V;
  for (int k = threadIdx.x; k < n2; k += blockDim.x)
    ((V*)A.out)[(int64_t)r * n2 + k] = make_pair_of<TS>(sm[k].x * inv, sm[k].y * inv);
}

template <typename TS>
void spectrum_launch(const SpecArgs& a, cudaStream_t st) {
  const int n = 1 << a.logn;
  if (n <= a.nsmem) {
    size_t smem = (size_t)n * sizeof(double2);
    set_smem((const void*)spec_smem_kernel<TS>, smem);
    spec_smem_kernel<TS><<<1, kThreads, smem, st>>>(a);
    return;
  }
  Split sp = split_of(a.logn);
  int C = four_step_cols<double>(sp.logn1);
  size_t smem = (size_t)C * ((size_t)(1 << sp.logn1) + 1) * sizeof(double2);
  set_smem((const void*)spec_col_kernel, smem);
  spec_col_kernel<<<(1 << sp.logn2) / C, kThreads, smem, st>>>(a, sp.logn1, sp.logn2, C);
  size_t smem2 = (size_t)(1 << sp.logn2) * sizeof(double2);
  set_smem((const void*)spec_row_kernel<TS>, smem2);
  spec_row_kernel<TS><<<1 << sp.logn1, kThreads, smem2, st>>>(a, sp.logn1, sp.logn2);
}

// ------------------------------------------------------------------ convolution

// Pointwise product of spectrum values with a kernel spectrum in the same storage order
// (the op of fftr_middle): x[j] *= spec[pos0 + j].
template <typename V>
struct SpecMul {
  const V* __restrict__ spec;
  template <class X, class RR>
  __device__ __forceinline__ void operator()(int t, int pos0, X& x, RR) const {
    (void)t;
    static_for<0, RR::value>([&](auto JJ) {
      constexpr int j = decltype(JJ)::value;
      x[j] = cmul(x[j], spec[pos0 + j]);
    });
  }
};

// One block per pair; the whole length-n transform in shared memory.  The first forward
// pass reads the input half straight from global memory, the last forward pass, the
// product with the kernel spectrum and the first inverse pass run fused in registers, and
// the last inverse pass writes (mode 0: subtracts) the wanted half straight to global.
template <typename T>
__global__ void __launch_bounds__(kThreads) conv_smem_kernel(ConvArgs A) {
  typedef Vt<T> V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int logn = A.logn, s = 1 << (logn - 1);
  const int64_t p = blockIdx.x;
  const V* __restrict__ zin = (const V*)A.zin + p * A.ld_in + A.in_off;
  V* __restrict__ zo = (V*)A.zout + p * A.ld_out + A.out_off;
  const V* __restrict__ tw = (const V*)A.tw;
  const SmLayout L = sm_layout<V>(logn);
  const int np = fftr_npasses<V>(logn);
  fftr_pass<V, true>(0, logn, 1, tw, true, [&](int, int e) { return zin[e]; }, SmPut<V>{sm, L});
  __syncthreads();
  if (np < 2) {  // a single pass: plain product in shared memory
    for (int k = threadIdx.x; k < 2 * s; k += blockDim.x) {
      const int q = sm_pos<V>(L, 0, k);
      sm[q] = cmul(sm[q], ((const V*)A.spec)[k]);
    }
    __syncthreads();
  } else {
    fftr_passes<V, true>(sm, logn, 1, tw, 1, np - 1, false);
    fftr_middle<V>(sm, logn, 1, SpecMul<V>{(const V*)A.spec});
    __syncthreads();
    fftr_passes<V, false>(sm, logn, 1, tw, 1, np - 1, false);
  }
  if (A.mode == 0) {
    fftr_pass<V, false>(np - 1, logn, 1, tw, false, SmAt<V>{sm, L}, [&](int, int e, const V& v) {
      if (e >= s) zo[e - s] = csub(zo[e - s], v);
    });
  } else {
    fftr_pass<V, false>(np - 1, logn, 1, tw, false, SmAt<V>{sm, L}, [&](int, int e, const V& v) {
      if (e < s) zo[e] = v;
    });
  }
}

// Four-step: n = n1*n2, index j = j1*n2 + j2.  Step A transforms C columns (over j1) per
// block, applies W_n^{j2 k1} and writes the scratch; step B transforms `rows` rows (over
// j2) per block, multiplies by the spectrum (stored in the same order), inverts the rows
// and removes the twiddle; step C inverts the columns.  Column transforms leave k1 in
// bit-reversed row order, which the twiddles account for.  Column kernels map consecutive
// threads to consecutive columns (coalesced global access); the first and last passes of
// every kernel read or write global memory directly.
template <typename T>
__global__ void __launch_bounds__(kThreads) conv_col_fwd_kernel(ConvArgs A, int logn1, int logn2, int C) {
  typedef Vt<T> V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int n2 = 1 << logn2, logn = logn1 + logn2, n = 1 << logn;
  const int c0 = blockIdx.x * C;
  const int64_t p = blockIdx.y;
  const V* __restrict__ zin = (const V*)A.zin + p * A.ld_in + A.in_off + c0;
  V* __restrict__ sc = (V*)A.scratch + p * (int64_t)n + c0;
  const V* __restrict__ tw = (const V*)A.tw;
  const V* __restrict__ twn = tw + (n - 2);
  const SmLayout L = sm_layout<V>(logn1);
  const int np = fftr_npasses<V>(logn1);
  fftr_pass<V, true, true>(0, logn1, C, tw, true, [&](int t, int e) { return zin[(int64_t)e * n2 + t]; },
                           SmPut<V>{sm, L});
  __syncthreads();
  fftr_passes<V, true, true>(sm, logn1, C, tw, 1, np - 1, false);
  fftr_pass<V, true, true>(np - 1, logn1, C, tw, false, SmAt<V>{sm, L}, [&](int t, int e, const V& v) {
    const int k1 = brev(e, logn1);
    sc[(int64_t)e * n2 + t] = cmul(v, twn[((int64_t)(c0 + t) * k1) & (n - 1)]);
  });
}

template <typename T>
__global__ void __launch_bounds__(kThreads) conv_row_kernel(ConvArgs A, int logn1, int logn2, int rows) {
  typedef Vt<T> V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int n2 = 1 << logn2, logn = logn1 + logn2, n = 1 << logn;
  const int r0 = blockIdx.x * rows;
  const int64_t p = blockIdx.y;
  V* __restrict__ sc = (V*)A.scratch + p * (int64_t)n + (int64_t)r0 * n2;
  const V* __restrict__ tw = (const V*)A.tw;
  const V* __restrict__ twn = tw + (n - 2);
  const SmLayout L = sm_layout<V>(logn2);
  const int np = fftr_npasses<V>(logn2);
  fftr_pass<V, true>(0, logn2, rows, tw, false, [&](int t, int e) { return sc[t * n2 + e]; }, SmPut<V>{sm, L});
  __syncthreads();
  fftr_passes<V, true>(sm, logn2, rows, tw, 1, np - 1, false);
  const V* __restrict__ spec = (const V*)A.spec + (int64_t)r0 * n2;
  fftr_middle<V>(sm, logn2, rows, [&](int t, int pos0, auto& x, auto RR) {
    SpecMul<V>{spec + t * n2}(t, pos0, x, RR);
  });
  __syncthreads();
  fftr_passes<V, false>(sm, logn2, rows, tw, 1, np - 1, false);
  fftr_pass<V, false>(np - 1, logn2, rows, tw, false, SmAt<V>{sm, L}, [&](int t, int e, const V& v) {
    const int k1 = brev(r0 + t, logn1);
    sc[t * n2 + e] = cmulc(v, twn[((int64_t)e * k1) & (n - 1)]);
  });
}

template <typename T>
__global__ void __launch_bounds__(kThreads) conv_col_inv_kernel(ConvArgs A, int logn1, int logn2, int C) {
  typedef Vt<T> V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int n2 = 1 << logn2, logn = logn1 + logn2, n = 1 << logn, h1 = 1 << (logn1 - 1);
  const int c0 = blockIdx.x * C;
  const int64_t p = blockIdx.y;
  const V* __restrict__ sc = (const V*)A.scratch + p * (int64_t)n + c0;
  V* __restrict__ zo = (V*)A.zout + p * A.ld_out + A.out_off + c0;
  const V* __restrict__ tw = (const V*)A.tw;
  const SmLayout L = sm_layout<V>(logn1);
  const int np = fftr_npasses<V>(logn1);
  fftr_pass<V, false, true>(0, logn1, C, tw, false, [&](int t, int e) { return sc[(int64_t)e * n2 + t]; },
                            SmPut<V>{sm, L});
  __syncthreads();
  fftr_passes<V, false, true>(sm, logn1, C, tw, 1, np - 1, false);
  if (A.mode == 0) {
    fftr_pass<V, false, true>(np - 1, logn1, C, tw, false, SmAt<V>{sm, L}, [&](int t, int e, const V& v) {
      if (e >= h1) {
        V* q = zo + (int64_t)(e - h1) * n2 + t;
        *q = csub(*q, v);
      }
    });
  } else {
    fftr_pass<V, false, true>(np - 1, logn1, C, tw, false, SmAt<V>{sm, L}, [&](int t, int e, const V& v) {
      if (e < h1) zo[(int64_t)e * n2 + t] = v;
    });
  }
}

// Columns per block of the four-step column kernels (power of two): 128-byte row
// segments, at most 64 KB of shared memory.
template <typename T>
int fourstep_cols(int logn1, int logn2) {
  int C = 128 / (int)sizeof(Vt<T>);
  while (C > 2 && (size_t)C * ((size_t)1 << logn1) * sizeof(Vt<T>) > 64 * 1024) C >>= 1;
  while (C > 1 && C > (1 << logn2)) C >>= 1;
  return C;
}
// Rows per block of the row kernel: about 16 elements per thread per pass.
template <typename T>
int fourstep_rows(int logn1, int logn2) {
  const int per = kThreads * (1 << EngineTraitsHost<T>::RB);
  int rows = per >> logn2;
  if (rows < 1) rows = 1;
  if (rows > (1 << logn1)) rows = 1 << logn1;
  return rows;
}

template <typename T>
void conv_launch(const ConvArgs& a, cudaStream_t st) {
  const int n = 1 << a.logn;
  if (n <= a.nsmem) {
    size_t smem = (size_t)n * sizeof(Vt<T>);
    set_smem((const void*)conv_smem_kernel<T>, smem);
    conv_smem_kernel<T><<<(unsigned)a.npairs, kThreads, smem, st>>>(a);
    return;
  }
  Split sp = split_of(a.logn);
  const int C = fourstep_cols<T>(sp.logn1, sp.logn2);
  const int rows = fourstep_rows<T>(sp.logn1, sp.logn2);
  const size_t smc = (size_t)C * ((size_t)1 << sp.logn1) * sizeof(Vt<T>);
  const size_t smr = (size_t)rows * ((size_t)1 << sp.logn2) * sizeof(Vt<T>);
  dim3 gc((unsigned)((1 << sp.logn2) / C), (unsigned)a.npairs);
  dim3 gr((unsigned)((1 << sp.logn1) / rows), (unsigned)a.npairs);
  set_smem((const void*)conv_col_fwd_kernel<T>, smc);
  set_smem((const void*)conv_row_kernel<T>, smr);
  set_smem((const void*)conv_col_inv_kernel<T>, smc);
  conv_col_fwd_kernel<T><<<gc, kThreads, smc, st>>>(a, sp.logn1, sp.logn2, C);
  conv_row_kernel<T><<<gr, kThreads, smr, st>>>(a, sp.logn1, sp.logn2, rows);
  conv_col_inv_kernel<T><<<gc, kThreads, smc, st>>>(a, sp.logn1, sp.logn2, C);
}

}  // namespace

int nsmem_for(Prec prec) { return prec == P32 ? 8192 : 4096; }
int bluestein_max_K(Prec prec) { return prec == P64 ? 2048 : 4096; }

int launch_dst_forward(Prec prec, const DstArgs& a, cudaStream_t st) {
  if (prec == P64) dst_launch<double>(a, true, st); else dst_launch<float>(a, true, st);
  return 1;
}
int launch_dst_inverse(Prec prec, const DstArgs& a, cudaStream_t st) {
  if (prec == P64) dst_launch<double>(a, false, st); else dst_launch<float>(a, false, st);
  return 1;
}

int launch_pack(Prec prec, const PackArgs& a, cudaStream_t st) {
  dim3 grid((unsigned)((a.ld + kThreads - 1) / kThreads), (unsigned)((a.nlines + 1) / 2));
  if (prec == P64) pack_kernel<double><<<grid, kThreads, 0, st>>>(a);
  else if (prec == P32) pack_kernel<float><<<grid, kThreads, 0, st>>>(a);
  else pack_kernel<FF><<<grid, kThreads, 0, st>>>(a);
  return 1;
}
int launch_unpack(Prec prec, const PackArgs& a, cudaStream_t st) {
  dim3 grid((unsigned)((a.N + kThreads - 1) / kThreads), (unsigned)((a.nlines + 1) / 2));
  if (prec == P64) unpack_kernel<double><<<grid, kThreads, 0, st>>>(a);
  else if (prec == P32) unpack_kernel<float><<<grid, kThreads, 0, st>>>(a);
  else unpack_kernel<FF><<<grid, kThreads, 0, st>>>(a);
  return 1;
}

int launch_scan(const ScanArgs& a, cudaStream_t st) {
  scan_kernel<<<(unsigned)a.M, kThreads, 0, st>>>(a);
  return 1;
}

int launch_residual(const ResidualArgs& a, cudaStream_t st) {
  dim3 grid((unsigned)((a.N + kThreads - 1) / kThreads), (unsigned)a.M);
  residual_kernel<<<grid, kThreads, 0, st>>>(a);
  return 1;
}

int launch_dot(const DotArgs& a, cudaStream_t st) {
  dot_kernel<<<a.nblocks, kThreads, 0, st>>>(a);
  return 1;
}
int launch_sum(const double* partial, int n, double* out, cudaStream_t st) {
  sum_kernel<<<1, kThreads, 0, st>>>(partial, n, out);
  return 1;
}

int launch_spectrum(Prec prec, const SpecArgs& a, cudaStream_t st) {
  if (prec == P64) spectrum_launch<double>(a, st);
  else if (prec == P32) spectrum_launch<float>(a, st);
  else spectrum_launch<FF>(a, st);
  return (1 << a.logn) <= a.nsmem ? 1 : 2;
}

int launch_conv(Prec prec, const ConvArgs& a, cudaStream_t st) {
  if (prec == P64) conv_launch<double>(a, st);
  else if (prec == P32) conv_launch<float>(a, st);
  else conv_launch<FF>(a, st);
  return (1 << a.logn) <= a.nsmem ? 1 : 3;
}

}  // namespace ftoep
