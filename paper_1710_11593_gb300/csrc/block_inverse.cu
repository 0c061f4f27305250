// Block solve by the inverse of the block operator: the per-level kernel (one block per
// pair, one time block per launch), the construction of the packed block-inverse spectra,
// and the unit impulse from which the substitution kernel of block_solve.cu builds the
// inverse first columns h_m once per plan.  The body and its derivation are in
// block_inverse_body.cuh.
#include "block_inverse_body.cuh"
#include "internal.h"

namespace ftoep {

namespace {

constexpr int kThreads = 256;

inline void set_smem(const void* fn, size_t bytes) { set_smem_once(fn, bytes); }

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

template <typename T>
__global__ void __launch_bounds__(kThreads, 3) block_inverse_kernel(BlockInvArgs A) {
  typedef Vt<T> V;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ T red[4 * kThreads];
  const int64_t p = blockIdx.x;
  const int n = 2 * A.B;
  block_inverse_body<T>(reinterpret_cast<V*>(smraw), (V*)A.z + p * A.ld + A.t0, (const V*)A.c1 + p * (int64_t)n,
                        A.logB, A.lamtau[p], A.prefix[p], red, A.prefix + p, (const V*)A.tw);
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
