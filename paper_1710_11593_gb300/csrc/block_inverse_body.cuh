// Device body of the block solve by the inverse of the block operator, shared by the
// per-level kernel (block_inverse.cu: one block per pair and time block) and the
// persistent per-pair solve (chain.cu).
//
// Every time block [t0, t0+B) of mode m solves the same system: the leading B x B
// principal submatrix of the lower-triangular Toeplitz operator T_m (difference form:
// E + lambda_m tau 1).  Its inverse is lower-triangular Toeplitz too, with first column
// h_m = the first B entries of T_m^-1 e_1, so the block solve is one causal convolution
//     x_b = h_m * (y_b - history),
// with the history of earlier blocks already subtracted by the cross-block updates except
// for the all-ones part, which is the constant lambda_m tau * (sum of all earlier x).
// The convolution is a cyclic one of length 2B, exact for outputs [0, B).
//
// Two modes with different kernels share one complex FFT: with Z = FFT(x_a + i x_b),
//     FFT(h_a * x_a) + i FFT(h_b * x_b) = C1 Z + C2 conj(Z_partner),
//     C1 = (H_a + H_b)/2, C2 = (H_a - H_b)/2,  partner of frequency k: n - k.
// C1 and C2 are spectra of real sequences, so C(n-k) = conj(C(k)); one length-2B array
// holds both (C1 at the lower of two partner positions, C2 at the other; the two
// self-partner frequencies 0 and n/2 share their slot as (C1, C2)).
#pragma once

#include "conv_body.cuh"

namespace ftoep {
namespace {

// Storage position of the partner (n - k mod n) of the frequency stored at `pos`
// (bit-reversed storage of a decimation-in-frequency FFT of length n = 2^logn).
__device__ __forceinline__ int partner_pos(int pos, int logn) {
  const int n = 1 << logn;
  const int k = brev(pos, logn);
  return brev((n - k) & (n - 1), logn);
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

// Block solve of one pair on one time block, in place: zg = the block's B entries of the
// pair row (right-hand side minus the cross-block history in, solution out), cs = the
// pair's packed C1/C2 array (2B entries), lt = lambda tau of the two modes, S = running
// sums of all earlier solved entries.  red: 4 * blockDim.x elements of shared memory.
// Thread 0 writes S advanced by this block's sums to *S_out.  No barrier at the end.
// ASYNC: the block's right-hand side arrives by cp.async into shared memory and the first
// pass (with the shift by the all-ones part) runs there.
template <typename T, int INF = 8, bool ASYNC = false>
__device__ __forceinline__ void block_inverse_body(Vt<T>* sm, Vt<T>* __restrict__ zg, const Vt<T>* __restrict__ cs,
                                                   int logB, double2 lt, double2 S, T* red, double2* S_out,
                                                   const Vt<T>* __restrict__ tw) {
  typedef Vt<T> V;
  const int B = 1 << logB, logn = logB + 1, n = 2 * B;
  const double sx = lt.x * S.x, sy = lt.y * S.y;
  const T sxh = (T)sx, syh = (T)sy;
  const T sxl = (T)(sx - (double)sxh), syl = (T)(sy - (double)syh);
  const SmLayout L = sm_layout<V>(logn);
  const int np = fftr_npasses<V>(logn);
  if constexpr (ASYNC) {
    for (int e = threadIdx.x; e < B; e += blockDim.x) async_copy(&sm[sm_pos<V>(L, 0, e)], zg + e);
    async_wait_all();
    fftr_pass<V, true>(0, logn, 1, tw, true, [&](int, int e) {
      const V y = sm[sm_pos<V>(L, 0, e)];
      return mkv(shift_sub(y.x, sxh, sxl), shift_sub(y.y, syh, syl));
    }, SmPut<V>{sm, L});
  } else {
    fftr_pass<V, true, false, true, false, INF>(0, logn, 1, tw, true, [&](int, int e) {
      const V y = zg[e];
      return mkv(shift_sub(y.x, sxh, sxl), shift_sub(y.y, syh, syl));
    }, SmPut<V>{sm, L});
  }
  __syncthreads();
  fftr_passes<V, true>(sm, logn, 1, tw, 1, np, false);
  // The product visits every frequency with its partner.  The pair's coefficients come
  // from global memory (64 KB per pair in float, read once per time block), so each thread
  // first issues the loads of kProdBatch of its positions, then does their arithmetic:
  // the loads of a batch are in flight together instead of one loop iteration at a time.
  constexpr int kProdBatch = 4;
  const int stride = blockDim.x;
  for (int base = threadIdx.x; base < n; base += kProdBatch * stride) {
    V c1v[kProdBatch], c2v[kProdBatch];
    int pv[kProdBatch], ppv[kProdBatch];
#pragma unroll
    for (int q = 0; q < kProdBatch; ++q) {
      const int pos = base + q * stride;
      pv[q] = pos;
      ppv[q] = pos < n ? partner_pos(pos, logn) : -1;
      if (pos < n && ppv[q] >= pos) {
        c1v[q] = cs[pos];
        c2v[q] = ppv[q] == pos ? c1v[q] : cs[ppv[q]];
      }
    }
#pragma unroll
    for (int q = 0; q < kProdBatch; ++q) {
      const int pos = pv[q], pp = ppv[q];
      if (pos >= n || pp < pos) continue;
      const int q1 = sm_pos<V>(L, 0, pos);
      const V z1 = sm[q1];
      V z1c;
      z1c.x = z1.x;
      z1c.y = -z1.y;
      if (pp == pos) {  // real C1, C2 packed in one slot
        const V c = c1v[q];
        V r;
        r.x = c.x * z1.x + c.y * z1c.x;
        r.y = c.x * z1.y + c.y * z1c.y;
        sm[q1] = r;
      } else {
        const V c1 = c1v[q], c2 = c2v[q];
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
  const int nt = blockDim.x;
  red[threadIdx.x] = ax;
  red[nt + threadIdx.x] = ay;
  red[2 * nt + threadIdx.x] = cx;
  red[3 * nt + threadIdx.x] = cy;
  __syncthreads();
  if (threadIdx.x < 32) {
    double tx = 0.0, ty = 0.0;
    for (int k = threadIdx.x; k < nt; k += 32) {
      tx += (double)red[k] + (double)red[2 * nt + k];
      ty += (double)red[nt + k] + (double)red[3 * nt + k];
    }
    for (int o = 16; o > 0; o >>= 1) {
      tx += __shfl_xor_sync(0xffffffffu, tx, o);
      ty += __shfl_xor_sync(0xffffffffu, ty, o);
    }
    if (threadIdx.x == 0) *S_out = make_double2(S.x + tx, S.y + ty);
  }
}

}  // namespace
}  // namespace ftoep
