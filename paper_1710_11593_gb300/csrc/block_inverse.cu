// Block solve by the inverse of the block operator.
//
// Every time block [t0, t0+B) of mode m solves the same system: the leading B x B
// principal submatrix of the lower-triangular Toeplitz operator T_m (difference form:
// E + lambda_m tau 1).  Its inverse is lower-triangular Toeplitz too, with first column
// h_m = the first B entries of T_m^-1 e_1, so the block solve is one causal convolution
//     x_b = h_m * (y_b - history),
// with the history of earlier blocks already subtracted by the cross-block updates except
// for the all-ones part, which is the constant lambda_m tau * (sum of all earlier x).
// h_m is computed once per plan (by the substitution kernel of block_solve.cu); the
// convolution is a cyclic one of length 2B, exact for outputs [0, B).
//
// Two modes with different kernels share one complex FFT: with Z = FFT(x_a + i x_b),
//     FFT(h_a * x_a) + i FFT(h_b * x_b) = C1 Z + C2 conj(Z_partner),
//     C1 = (H_a + H_b)/2, C2 = (H_a - H_b)/2,  partner of frequency k: n - k,
// and H_a, H_b themselves are split out of FFT(h_a + i h_b) the same way.
#include "fft.cuh"
#include "internal.h"

namespace ftoep {

namespace {

constexpr int kThreads = 256;

template <typename T>
using Vt = typename VecOf<T>::type;

inline void set_smem(const void* fn, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Storage position of the partner (n - k mod n) of the frequency stored at `pos`
// (bit-reversed storage of a decimation-in-frequency FFT of length n = 2^logn).
__device__ __forceinline__ int partner_pos(int pos, int logn) {
  const int n = 1 << logn;
  const int k = brev(pos, logn);
  return brev((n - k) & (n - 1), logn);
}

__global__ void unit_impulse_kernel(double2* z, int64_t ld, int64_t npairs, int B) {
  const int64_t p = blockIdx.x;
  if (p >= npairs) return;
  for (int i = threadIdx.x; i < B; i += blockDim.x) z[p * ld + i] = i == 0 ? make_double2(1.0, 1.0) : make_double2(0.0, 0.0);
}

template <typename TS>
__global__ void __launch_bounds__(kThreads) inverse_spectrum_kernel(InvSpecArgs A) {
  typedef Vt<TS> VS;
  extern __shared__ __align__(16) unsigned char smraw[];
  double2* sm = reinterpret_cast<double2*>(smraw);
  const int B = A.B, logn = A.logB + 1, n = 2 * B;
  const int64_t p = blockIdx.x;
  const double2* h = A.h + p * A.ldh;
  for (int i = threadIdx.x; i < B; i += blockDim.x) sm[i] = h[i];
  __syncthreads();
  fft_dif<double2>(sm, logn, 1, 0, A.tw64, true);
  const double inv = 1.0 / (double)n;
  VS* c1 = (VS*)A.c1 + p * (int64_t)n;
  VS* c2 = (VS*)A.c2 + p * (int64_t)n;
  for (int pos = threadIdx.x; pos < n; pos += blockDim.x) {
    const double2 zk = sm[pos];
    const double2 zp = sm[partner_pos(pos, logn)];
    // H_a = (Zk + conj Zp)/2, H_b = (Zk - conj Zp)/(2i)
    const double har = 0.5 * (zk.x + zp.x), hai = 0.5 * (zk.y - zp.y);
    const double hbr = 0.5 * (zk.y + zp.y), hbi = -0.5 * (zk.x - zp.x);
    c1[pos] = mkv((TS)(0.5 * (har + hbr) * inv), (TS)(0.5 * (hai + hbi) * inv));
    c2[pos] = mkv((TS)(0.5 * (har - hbr) * inv), (TS)(0.5 * (hai - hbi) * inv));
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) block_inverse_kernel(BlockInvArgs A) {
  typedef Vt<T> V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  __shared__ double red[2][kThreads / 32];
  const int B = A.B, logn = A.logB + 1, n = 2 * B;
  const int64_t p = blockIdx.x;
  V* zg = (V*)A.z + p * A.ld + A.t0;
  const double2 S = A.prefix[p];
  const double2 lt = A.lamtau[p];
  const double sx = lt.x * S.x, sy = lt.y * S.y;
  for (int i = threadIdx.x; i < B; i += blockDim.x) {
    const V y = zg[i];
    sm[i] = mkv((T)((double)y.x - sx), (T)((double)y.y - sy));
  }
  __syncthreads();
  const V* tw = (const V*)A.tw;
  fft_dif<V>(sm, logn, 1, 0, tw, true);
  const V* c1 = (const V*)A.c1 + p * (int64_t)n;
  const V* c2 = (const V*)A.c2 + p * (int64_t)n;
  for (int pos = threadIdx.x; pos < n; pos += blockDim.x) {
    const int pp = partner_pos(pos, logn);
    if (pp < pos) continue;
    const V z1 = sm[pos];
    if (pp == pos) {
      V zc;
      zc.x = z1.x;
      zc.y = -z1.y;
      sm[pos] = cadd(cmul(c1[pos], z1), cmul(c2[pos], zc));
    } else {
      const V z2 = sm[pp];
      V z1c, z2c;
      z1c.x = z1.x;
      z1c.y = -z1.y;
      z2c.x = z2.x;
      z2c.y = -z2.y;
      sm[pos] = cadd(cmul(c1[pos], z1), cmul(c2[pos], z2c));
      sm[pp] = cadd(cmul(c1[pp], z2), cmul(c2[pp], z1c));
    }
  }
  __syncthreads();
  fft_dit<V>(sm, logn, 1, 0, tw, 2);
  double ax = 0.0, ay = 0.0;
  for (int i = threadIdx.x; i < B; i += blockDim.x) {
    const V x = sm[i];
    zg[i] = x;
    ax += (double)x.x;
    ay += (double)x.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    ax += __shfl_xor_sync(0xffffffffu, ax, o);
    ay += __shfl_xor_sync(0xffffffffu, ay, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = ax;
    red[1][threadIdx.x >> 5] = ay;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tx = 0.0, ty = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) {
      tx += red[0][w];
      ty += red[1][w];
    }
    A.prefix[p] = make_double2(S.x + tx, S.y + ty);
  }
}

template <typename T>
void inverse_launch(const BlockInvArgs& a, cudaStream_t st) {
  const size_t smem = (size_t)2 * a.B * sizeof(Vt<T>);
  set_smem((const void*)block_inverse_kernel<T>, smem);
  block_inverse_kernel<T><<<(unsigned)a.npairs, kThreads, smem, st>>>(a);
}

}  // namespace

int launch_unit_impulse(double2* z, int64_t ld, int64_t npairs, int B, cudaStream_t st) {
  unit_impulse_kernel<<<(unsigned)npairs, kThreads, 0, st>>>(z, ld, npairs, B);
  return 1;
}

int launch_inverse_spectrum(Prec prec, const InvSpecArgs& a, cudaStream_t st) {
  const size_t smem = (size_t)2 * a.B * sizeof(double2);
  if (prec == P64) {
    set_smem((const void*)inverse_spectrum_kernel<double>, smem);
    inverse_spectrum_kernel<double><<<(unsigned)a.npairs, kThreads, smem, st>>>(a);
  } else {
    set_smem((const void*)inverse_spectrum_kernel<float>, smem);
    inverse_spectrum_kernel<float><<<(unsigned)a.npairs, kThreads, smem, st>>>(a);
  }
  return 1;
}

int launch_block_inverse(Prec prec, const BlockInvArgs& a, cudaStream_t st) {
  if (prec == P64) inverse_launch<double>(a, st); else inverse_launch<float>(a, st);
  return 1;
}

}  // namespace ftoep
