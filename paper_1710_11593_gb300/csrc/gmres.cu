// Vector kernels of the restarted GMRES method of Sec. 3.2 and of the advection sweeps of Sec. 3
// (the right-hand sides of all nodes, one round of the scan over the nodes).
//
// GMRES: the method of Sec. 3.2 (Saad and Schultz, as the paper
// states it) on the space-time systems of the reordered schemes (Eq. 21: block rows A-hat on
// the diagonal, B-hat = -1/h^2 I beside it, i.e. I_M (x) T + K (x) I_N with T the time
// operator's lower-triangular Toeplitz matrix and K the spatial second difference).  The
// Toeplitz part of every product runs through the library's circulant-embedded product
// (Sec. 3.1, Eq. be1); these kernels add the spatial part and carry the Arnoldi process.
// Fields are [M][N] doubles, time contiguous.
#include "internal.h"

namespace ftoep {

namespace {

constexpr int kThreads = 256;

// y += S x, S the spatial operator of the left-hand side: (2x_j - x_{j-1} - x_{j+1})/h^2
// (space 1, zero boundary values) or lambda x_j (space 0), applied with weight sw at time
// level n and 1 - sw at level n-1 (sw = 1/2: the Crank-Nicolson average; x at level 0 is
// zero -- the systems carry zero initial data).
__global__ void space_add_kernel(double* __restrict__ y, const double* __restrict__ x, int64_t M, int64_t N,
                                 int space, double inv_h2, double lambda, double sw) {
  const int64_t total = M * N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / N, n = e % N;
    auto S = [&](int64_t col) -> double {
      const double c = x[j * N + col];
      if (space == 0) return lambda * c;
      const double l = j > 0 ? x[(j - 1) * N + col] : 0.0;
      const double r = j + 1 < M ? x[(j + 1) * N + col] : 0.0;
      return (2.0 * c - l - r) * inv_h2;
    };
    double s = sw * S(n);
    if (sw != 1.0 && n > 0) s += (1.0 - sw) * S(n - 1);
    y[e] += s;
  }
}

// partial[i * gridDim.x + b] = block b's part of <V_i, w>, i = blockIdx.y < k.
__global__ void mdot_kernel(const double* __restrict__ V, int64_t ldv, const double* __restrict__ w, int64_t L,
                            double* __restrict__ partial) {
  __shared__ double red[kThreads / 32];
  const double* v = V + (int64_t)blockIdx.y * ldv;
  double acc = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < L; e += (int64_t)gridDim.x * blockDim.x)
    acc = fma(v[e], w[e], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    partial[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

// w += sum_{i<k} c_i V_i  (k <= kMaxBasis, coefficients in device memory).
__global__ void maxpy_kernel(double* __restrict__ w, const double* __restrict__ V, int64_t ldv, int k,
                             const double* __restrict__ c, int64_t L) {
  __shared__ double cs[kMaxBasis];
  for (int i = threadIdx.x; i < k; i += blockDim.x) cs[i] = c[i];
  __syncthreads();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < L; e += (int64_t)gridDim.x * blockDim.x) {
    double acc = w[e];
    for (int i = 0; i < k; ++i) acc = fma(cs[i], V[(int64_t)i * ldv + e], acc);
    w[e] = acc;
  }
}

// y = a x + b z (y may be x: no restrict qualifiers)
__global__ void lincomb_kernel(double* y, double a, const double* x, double b, const double* z, int64_t L) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < L; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = a * x[e] + (b != 0.0 ? b * z[e] : 0.0);
}

// Right-hand sides of all nodes of an advection sweep: g[i][n] = c F[i][n] + s0[i] w0[n] +
// s1[i] w1[n] (w0/s0, w1/s1 nullable).
__global__ void sweep_rhs_lines_kernel(double* __restrict__ g, const double* __restrict__ F,
                                       const double* __restrict__ w0, const double* __restrict__ s0,
                                       const double* __restrict__ w1, const double* __restrict__ s1, int64_t M,
                                       int64_t N, double c) {
  const int64_t total = M * N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / N, n = e % N;
    double v = c * F[e];
    if (w0) v = fma(s0[i], w0[n], v);
    if (w1) v = fma(s1[i], w1[n], v);
    g[e] = v;
  }
}

// One round of the space scan: out[i] = in[i] + t[i - d] for i >= d, out[i] = in[i] below.
__global__ void shift_add_lines_kernel(double* __restrict__ out, const double* __restrict__ in,
                                       const double* __restrict__ t, int64_t M, int64_t N, int64_t d) {
  const int64_t total = M * N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / N;
    out[e] = i >= d ? in[e] + t[e - d * N] : in[e];
  }
}

unsigned grid_for(int64_t L) {
  const int64_t b = (L + kThreads - 1) / kThreads;
  return (unsigned)std::min<int64_t>(std::max<int64_t>(b, 1), 152 * 8);
}

}  // namespace

int launch_space_add(double* y, const double* x, int64_t M, int64_t N, int space, double inv_h2, double lambda,
                     double sw, cudaStream_t st) {
  space_add_kernel<<<grid_for(M * N), kThreads, 0, st>>>(y, x, M, N, space, inv_h2, lambda, sw);
  return 1;
}

int launch_mdot(const double* V, int64_t ldv, int k, const double* w, int64_t L, double* partial, int nblocks,
                cudaStream_t st) {
  mdot_kernel<<<dim3((unsigned)nblocks, (unsigned)k), kThreads, 0, st>>>(V, ldv, w, L, partial);
  return 1;
}

int launch_maxpy(double* w, const double* V, int64_t ldv, int k, const double* c, int64_t L, cudaStream_t st) {
  maxpy_kernel<<<grid_for(L), kThreads, 0, st>>>(w, V, ldv, k, c, L);
  return 1;
}

int launch_sweep_rhs_lines(double* g, const double* F, const double* w0, const double* s0, const double* w1,
                           const double* s1, int64_t M, int64_t N, double c, cudaStream_t st) {
  sweep_rhs_lines_kernel<<<grid_for(M * N), kThreads, 0, st>>>(g, F, w0, s0, w1, s1, M, N, c);
  return 1;
}

int launch_shift_add_lines(double* out, const double* in, const double* t, int64_t M, int64_t N, int64_t d,
                           cudaStream_t st) {
  shift_add_lines_kernel<<<grid_for(M * N), kThreads, 0, st>>>(out, in, t, M, N, d);
  return 1;
}

int launch_lincomb(double* y, double a, const double* x, double b, const double* z, int64_t L, cudaStream_t st) {
  lincomb_kernel<<<grid_for(L), kThreads, 0, st>>>(y, a, x, b, z, L);
  return 1;
}

}  // namespace ftoep
