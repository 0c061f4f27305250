// In-block half-split solve of the lower-triangular Toeplitz systems
//     (lambda_m I + T) x_m = y_m,   T first column a  (Sec. 3: the reordered per-line
// systems A-hat U_i = F_i; lambda_m from the sine decoupling of the spatial operator)
// on one time block [t0, t0+B) of every mode pair, with the history of earlier blocks
// already subtracted from y.
//
// Recursion on [lo, hi), mid = (lo+hi)/2:  solve [lo, mid);
//     y[mid, hi) -= T21 x[lo, mid),  (T21)_{ik} = a_{s+i-k},  s = mid - lo;
// solve [mid, hi).  Written iteratively: after leaf b (leaves of length L) the one update
// that becomes due has s = L * 2^ctz(b+1).  Leaves are forward substitutions in double
// precision; levels s < Sf are direct products (s^2 multiply-adds per component);
// levels s >= Sf are cyclic convolutions of length 2s in shared memory, exact for this
// block because the needed entries a_1 .. a_{2s-1} never wrap around.
//
// Used once per plan: applied to a unit impulse it yields the first B entries h_m of
// every mode's inverse block operator, from which block_inverse.cu builds the spectra
// of the block solve that the timed path uses.
#include "fft.cuh"
#include "internal.h"

namespace ftoep {

namespace {

constexpr int kThreads = 256;

template <typename T>
using Vt = typename VecOf<T>::type;

// Leaf forward substitution in double precision, one warp.  The operator of mode c is
// T_c = E + (lambda_c tau) 1, with E the shared lower-triangular Toeplitz matrix (first
// column e) and 1 the all-ones lower triangle.  The all-ones part couples a row to every
// earlier unknown through their sum, so the leaf receives the running sum P_c of all
// earlier unknowns and returns it advanced over its own L unknowns.  Unit-diagonal form,
// with d_c = e_0 + lambda_c tau:
//     y'_i = (y_i - lambda_c tau P_c)/d_c,  x_k = y'_k,  y'_i -= ((e_{i-k} + lambda_c tau)/d_c) x_k,
// one shuffle and one FMA per step.  Lane l = c*L + i (i < L <= 16) owns row i of
// component c (c = 0: mode 2p in .x, c = 1: mode 2p+1 in .y); asc[c*L + j] holds
// (e_j + lambda_c tau)/d_c and P (per lane, for its component) stays in a register.
template <typename T>
__device__ __forceinline__ void leaf_solve(Vt<T>* zb, int L, const double* asc, double inv, double lt, double& P) {
  const int lane = threadIdx.x;
  const int c = lane >= L ? 1 : 0;
  const int i = lane - c * L;
  const bool act = lane < 2 * L;
  double y = 0.0;
  if (act) {
    const Vt<T> z = zb[i];
    y = ((c ? (double)z.y : (double)z.x) - lt * P) * inv;
  }
  const double* ac = asc + c * L;
  for (int k = 0; k < L; ++k) {
    const double xk = __shfl_sync(0xffffffffu, y, c * L + k);
    if (act && i > k) y = fma(-ac[i - k], xk, y);
  }
  if (act) {
    if (c) zb[i].y = (T)y; else zb[i].x = (T)y;
  }
  // advance the running sum by this leaf's unknowns (segments of L lanes)
  double t = act ? y : 0.0;
  for (int w = 1; w < L; w <<= 1) t += __shfl_xor_sync(0xffffffffu, t, w);
  P += t;
}

// y[mid + i] -= sum_{k<s} a_{s+i-k} x[mid - s + k], both components, direct sums.
template <typename T>
__device__ __forceinline__ void dense_update(Vt<T>* zb, int mid, int s, const T* at) {
  const int nout = 2 * s;
  int G = kThreads / nout;
  if (G > 32) G = 32;
  if (G < 1) G = 1;
  const int ngroups = kThreads / G;
  const int g = threadIdx.x % G;
  for (int o0 = 0; o0 < nout; o0 += ngroups) {
    const int o = o0 + threadIdx.x / G;
    T acc = (T)0;
    if (o < nout) {
      const int i = o >> 1, comp = o & 1;
      const Vt<T>* xb = zb + (mid - s);
      for (int k = g; k < s; k += G) {
        const Vt<T> xv = xb[k];
        acc = fma(at[s + i - k], comp ? xv.y : xv.x, acc);
      }
    }
    for (int w = G >> 1; w > 0; w >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, w);
    if (o < nout && g == 0) {
      const int i = o >> 1;
      if (o & 1) zb[mid + i].y -= acc; else zb[mid + i].x -= acc;
    }
  }
}

template <typename T>
__device__ __forceinline__ void fft_update(Vt<T>* zb, Vt<T>* fb, int mid, int s, const Vt<T>* spec,
                                           const Vt<T>* tw) {
  typedef Vt<T> V;
  const int n = 2 * s;
  const int logn = __ffs(n) - 1;
  for (int i = threadIdx.x; i < s; i += blockDim.x) fb[i] = zb[mid - s + i];
  __syncthreads();
  fft_dif<V>(fb, logn, 1, 0, tw, true);
  for (int k = threadIdx.x; k < n; k += blockDim.x) fb[k] = cmul(fb[k], spec[k]);
  __syncthreads();
  fft_dit<V>(fb, logn, 1, 0, tw, 1);
  for (int i = threadIdx.x; i < s; i += blockDim.x) zb[mid + i] = csub(zb[mid + i], fb[s + i]);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) block_solve_kernel(BlockArgs A) {
  typedef Vt<T> V;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int B = A.B, L = A.L, Sf = A.Sf;
  V* zb = reinterpret_cast<V*>(smraw);
  V* fb = zb + B;
  const int nat = (2 * Sf < B) ? 2 * Sf : B;  // a_k needed by the dense levels: k < 2s <= 2*Sf
  double* asc = reinterpret_cast<double*>(fb + B);  // 2L scaled leaf coefficients
  T* at = reinterpret_cast<T*>(asc + 32);
  const int64_t p = blockIdx.x;
  V* zg = (V*)A.z + p * A.ld + A.t0;
  for (int i = threadIdx.x; i < B; i += blockDim.x) zb[i] = zg[i];
  for (int i = threadIdx.x; i < nat; i += blockDim.x) at[i] = (T)A.a[i];
  const double2 inv = A.invdiag[p];
  const double2 lt = A.lamtau[p];
  for (int i = threadIdx.x; i < 2 * L; i += blockDim.x) {
    const int j = i % L;
    asc[i] = j == 0 ? 0.0 : (A.a[j] + (i < L ? lt.x : lt.y)) * (i < L ? inv.x : inv.y);
  }
  // warp 0 carries the running sums: lanes of component 0 hold P.x, of component 1 P.y
  const bool c1lane = threadIdx.x >= L && threadIdx.x < 2 * L;
  double P = 0.0;
  if (threadIdx.x < 32) {
    const double2 p0 = A.prefix[p];
    P = c1lane ? p0.y : p0.x;
  }
  const double my_inv = c1lane ? inv.y : inv.x;
  const double my_lt = c1lane ? lt.y : lt.x;
  const V* spec = (const V*)A.spec;
  const V* tw = (const V*)A.tw;
  __syncthreads();
  const int nleaf = B / L;
  for (int b = 0; b < nleaf; ++b) {
    if (threadIdx.x < 32) leaf_solve<T>(zb + b * L, L, asc, my_inv, my_lt, P);
    __syncthreads();
    const int v = b + 1;
    if (v < nleaf) {
      const int s = L << (__ffs(v) - 1);
      const int mid = v * L;
      if (s < Sf) {
        dense_update<T>(zb, mid, s, at);
      } else {
        fft_update<T>(zb, fb, mid, s, spec + 2 * (s - Sf), tw);
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < B; i += blockDim.x) zg[i] = zb[i];
  if (threadIdx.x < 32) {
    const double py = __shfl_sync(0xffffffffu, P, L);
    if (threadIdx.x == 0) A.prefix[p] = make_double2(P, py);
  }
}

template <typename T>
size_t smem_bytes(int B, int Sf) {
  const int nat = (2 * Sf < B) ? 2 * Sf : B;
  return (size_t)B * 2 * sizeof(Vt<T>) + 32 * sizeof(double) + (size_t)nat * sizeof(T);
}

template <typename T>
void launch(const BlockArgs& a, cudaStream_t st) {
  const size_t smem = smem_bytes<T>(a.B, a.Sf);
  set_smem_once((const void*)block_solve_kernel<T>, smem);
  block_solve_kernel<T><<<(unsigned)a.npairs, kThreads, smem, st>>>(a);
}

}  // namespace

size_t block_solve_smem(Prec prec, int B, int Sf) {
  return prec == P64 ? smem_bytes<double>(B, Sf) : smem_bytes<float>(B, Sf);
}

int launch_block_solve(Prec prec, const BlockArgs& a, cudaStream_t st) {
  if (prec == P64) launch<double>(a, st); else launch<float>(a, st);
  return 1;
}

}  // namespace ftoep
