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
#include "fftr.cuh"
#include "internal.h"

namespace ftoep {

namespace {

constexpr int kThreads = 256;

template <typename T>
using Vt = typename VecOf<T>::type;

inline void set_smem(const void* fn, size_t bytes) { set_smem_once(fn, bytes); }

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

// C1 and C2 are spectra of real sequences ((h_a +- h_b)/2), so C(n-k) = conj(C(k)), and the
// solve visits every frequency together with its partner.  One length-n array holds both:
// at the position of the lower of the two partner positions C1, at the partner's position
// C2 of that lower one; the two self-partner frequencies (0 and n/2) are real and share
// their slot as (C1, C2).
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
  VS* c = (VS*)A.c1 + p * (int64_t)n;
  for (int pos = threadIdx.x; pos < n; pos += blockDim.x) {
    const int pp = partner_pos(pos, logn);
    const int lo = pos < pp ? pos : pp;
    const double2 zk = sm[lo];
    const double2 zp = sm[partner_pos(lo, logn)];
    // H_a = (Zk + conj Zp)/2, H_b = (Zk - conj Zp)/(2i) at the lower position
    const double har = 0.5 * (zk.x + zp.x), hai = 0.5 * (zk.y - zp.y);
    const double hbr = 0.5 * (zk.y + zp.y), hbi = -0.5 * (zk.x - zp.x);
    const double c1r = 0.5 * (har + hbr) * inv, c1i = 0.5 * (hai + hbi) * inv;
    const double c2r = 0.5 * (har - hbr) * inv, c2i = 0.5 * (hai - hbi) * inv;
    if (pos == pp) c[pos] = mkv((TS)c1r, (TS)c2r);
    else if (pos < pp) c[pos] = mkv((TS)c1r, (TS)c1i);
    else c[pos] = mkv((TS)c2r, (TS)c2i);
  }
}

// y - lambda tau S for one component: double arithmetic for the double path; for the
// float path S' = lambda tau S is split into a float pair (hi + lo) once per block, so the
// per-element work stays in FP32 (GB300 runs FP64 at 1/64 of the FP32 rate).
__device__ __forceinline__ double shift_sub(double y, double sh, double) { return y - sh; }
__device__ __forceinline__ float shift_sub(float y, float sh, float sl) { return (y - sh) - sl; }

// s + c += x with the rounding error of the addition kept in c (Knuth two-sum); the double
// path adds directly (c stays 0).
__device__ __forceinline__ void acc2(double& s, double&, double x) { s += x; }
__device__ __forceinline__ void acc2(float& s, float& c, float x) {
  const float t = s + x;
  const float bb = t - s;
  c += (s - (t - bb)) + (x - bb);
  s = t;
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 3) block_inverse_kernel(BlockInvArgs A) {
  typedef Vt<T> V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  __shared__ T red[4][kThreads];
  const int B = A.B, logn = A.logB + 1, n = 2 * B;
  const int64_t p = blockIdx.x;
  V* __restrict__ zg = (V*)A.z + p * A.ld + A.t0;
  const double2 S = A.prefix[p];
  const double2 lt = A.lamtau[p];
  const double sx = lt.x * S.x, sy = lt.y * S.y;
  const T sxh = (T)sx, syh = (T)sy;
  const T sxl = (T)(sx - (double)sxh), syl = (T)(sy - (double)syh);
  const V* __restrict__ tw = (const V*)A.tw;
  const SmLayout L = sm_layout<V>(logn);
  const int np = fftr_npasses<V>(logn);
  fftr_pass<V, true, false, true>(0, logn, 1, tw, true, [&](int, int e) {
    const V y = zg[e];
    return mkv(shift_sub(y.x, sxh, sxl), shift_sub(y.y, syh, syl));
  }, SmPut<V>{sm, L});
  __syncthreads();
  fftr_passes<V, true>(sm, logn, 1, tw, 1, np, false);
  const V* __restrict__ cs = (const V*)A.c1 + p * (int64_t)n;
  for (int pos = threadIdx.x; pos < n; pos += blockDim.x) {
    const int pp = partner_pos(pos, logn);
    if (pp < pos) continue;
    const int q1 = sm_pos<V>(L, 0, pos);
    const V z1 = sm[q1];
    V z1c;
    z1c.x = z1.x;
    z1c.y = -z1.y;
    if (pp == pos) {  // real C1, C2 packed in one slot
      const V c = cs[pos];
      V r;
      r.x = c.x * z1.x + c.y * z1c.x;
      r.y = c.x * z1.y + c.y * z1c.y;
      sm[q1] = r;
    } else {
      const V c1 = cs[pos], c2 = cs[pp];
      const int q2 = sm_pos<V>(L, 0, pp);
      const V z2 = sm[q2];
      V z2c;
      z2c.x = z2.x;
      z2c.y = -z2.y;
      // Y_k = C1_k Z_k + C2_k conj(Z_{n-k}); at the partner the conjugate coefficients
      sm[q1] = cadd(cmul(c1, z1), cmul(c2, z2c));
      sm[q2] = cadd(cmulc(z2, c1), cmulc(z1c, c2));
    }
  }
  __syncthreads();
  fftr_passes<V, false>(sm, logn, 1, tw, 0, np - 1, false);
  // block sums of x for the running prefix: compensated (two-sum) per thread, then the
  // per-thread pairs are added in double by one warp
  T ax = (T)0, ay = (T)0, cx = (T)0, cy = (T)0;
  fftr_pass<V, false>(np - 1, logn, 1, tw, false, SmAt<V>{sm, L}, [&](int, int e, const V& x) {
    if (e < B) {
      zg[e] = x;
      acc2(ax, cx, x.x);
      acc2(ay, cy, x.y);
    }
  });
  red[0][threadIdx.x] = ax;
  red[1][threadIdx.x] = ay;
  red[2][threadIdx.x] = cx;
  red[3][threadIdx.x] = cy;
  __syncthreads();
  if (threadIdx.x < 32) {
    double tx = 0.0, ty = 0.0;
    for (int k = threadIdx.x; k < kThreads; k += 32) {
      tx += (double)red[0][k] + (double)red[2][k];
      ty += (double)red[1][k] + (double)red[3][k];
    }
    for (int o = 16; o > 0; o >>= 1) {
      tx += __shfl_xor_sync(0xffffffffu, tx, o);
      ty += __shfl_xor_sync(0xffffffffu, ty, o);
    }
    if (threadIdx.x == 0) A.prefix[p] = make_double2(S.x + tx, S.y + ty);
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
