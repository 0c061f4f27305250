// Scheme 1 of the paper (Sec. 2): the two-sided fractional ODE
//     D_left^g u + D_right^g u + u = f  on (0, T),  u(0) = u(T) = 0,  0 < g < 1,
// discretised with the left L1 formula (Eq. 4) and the right one (Eq. 5) on tau = T/N: the
// system A u = f of Eq. 9 on u_1 .. u_{N-1}, A symmetric positive definite Toeplitz
// (Theorem 1) with first column
//     a_0 = 1 + 2 mu G_0,   a_d = mu (G_d - G_{d-1}) = mu W_d   (d = 1 .. N-2),
// mu = tau^-g / Gamma(2-g).  Solved by the conjugate gradient method of Sec. 2.3, every
// product A w by circulant embedding (Eq. 10): c = [a_0 .. a_{n-1}, 0 .., a_{n-1} .. a_1] of
// a power-of-two length L >= 2n (n = N-1), with the input padded by zeros (the printed
// (w, w) vector would add the wrong half, see the reading of the circulant vector), and the
// library's FFT convolution.  The iteration itself: residual and direction updates and the
// two inner products per iteration in double on the GPU, the scalars read back per
// iteration for the step lengths and the stopping test.
#include <cmath>
#include <cstdio>
#include <vector>

#include "../../include/ftoep.h"
#include "internal.h"

namespace ftoep {

namespace {

constexpr int kCgThreads = 256;
constexpr int kCgBlocks = 512;

// partial[b] = sum over the block's grid-stride share of x[i] * y[i]
__global__ void __launch_bounds__(kCgThreads) cg_dot_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                                             int64_t n, double* __restrict__ partial) {
  __shared__ double red[kCgThreads / 32];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s = fma(x[i], y[i], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kCgThreads / 32; ++w) t += red[w];
    partial[blockIdx.x] = t;
  }
}

// out[k] = sum of partial[k * nb .. (k+1) * nb), one block per k
__global__ void __launch_bounds__(kCgThreads) cg_sum_kernel(const double* __restrict__ partial, int nb,
                                                             double* __restrict__ out) {
  __shared__ double red[kCgThreads / 32];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += partial[(int64_t)blockIdx.x * nb + i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kCgThreads / 32; ++w) t += red[w];
    out[blockIdx.x] = t;
  }
}

// u += alpha w,  r -= alpha q
__global__ void cg_step_kernel(double* __restrict__ u, double* __restrict__ r, const double* __restrict__ w,
                               const double* __restrict__ q, double alpha, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    u[i] = fma(alpha, w[i], u[i]);
    r[i] = fma(-alpha, q[i], r[i]);
  }
}

// w = r + beta w
__global__ void cg_direction_kernel(double* __restrict__ w, const double* __restrict__ r, double beta, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    w[i] = fma(beta, w[i], r[i]);
}

// r = f - q
__global__ void cg_sub_kernel(double* __restrict__ r, const double* __restrict__ f, const double* __restrict__ q,
                              int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    r[i] = f[i] - q[i];
}

struct Cg {
  int64_t n = 0, L = 0;
  int logL = 0;
  cudaStream_t st = nullptr;
  std::vector<void*> mem;
  double *c = nullptr, *f = nullptr, *u = nullptr, *r = nullptr, *w = nullptr, *q = nullptr;
  double *partial = nullptr, *scal = nullptr;
  double2 *tw = nullptr, *spec = nullptr, *z = nullptr, *scratch = nullptr;
  ~Cg() {
    for (void* p : mem) cudaFree(p);
  }
  template <typename P>
  ftoep_status alloc(P** out, size_t bytes) {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      char buf[128];
      snprintf(buf, sizeof(buf), "ftoep_two_sided_cg: cudaMalloc(%zu bytes) failed", bytes);
      set_global_error(buf);
      return FTOEP_ENOMEM;
    }
    mem.push_back(p);
    *out = (P*)p;
    return FTOEP_OK;
  }
};

ftoep_status cuda_fail(const char* what) {
  const cudaError_t e = cudaGetLastError();
  char buf[256];
  snprintf(buf, sizeof(buf), "ftoep_two_sided_cg: %s: %s", what, cudaGetErrorString(e));
  set_global_error(buf);
  return FTOEP_ECUDA;
}

#define CG_TRY(expr)                     \
  do {                                   \
    ftoep_status s_ = (expr);            \
    if (s_ != FTOEP_OK) return s_;       \
  } while (0)
#define CG_CK(call, what)                                   \
  do {                                                      \
    if ((call) != cudaSuccess) return cuda_fail(what);      \
  } while (0)

// q = A x through the circulant embedding.
ftoep_status apply(Cg& g, const double* x, double* q) {
  PackArgs pa{};
  pa.x = x;
  pa.y = q;
  pa.z = g.z;
  pa.ld = g.L / 2;
  pa.N = g.n;
  pa.nlines = 1;
  launch_pack(P64, pa, g.st);
  ConvArgs ca{};
  ca.zin = g.z;
  ca.zout = g.z;
  ca.ld_in = ca.ld_out = g.L / 2;
  ca.npairs = 1;
  ca.logn = g.logL;
  ca.nsmem = nsmem_for(P64);
  ca.mode = 1;
  ca.spec = g.spec;
  ca.tw = g.tw;
  ca.scratch = g.scratch;
  launch_conv(P64, ca, g.st);
  pa.mode = 0;
  launch_unpack(P64, pa, g.st);
  if (cudaPeekAtLastError() != cudaSuccess) return cuda_fail("product launch");
  return FTOEP_OK;
}

// host[0..k) = <x_i, y_i> for the k pairs
ftoep_status dots(Cg& g, const double* const* xs, const double* const* ys, int k, double* host) {
  for (int i = 0; i < k; ++i)
    cg_dot_kernel<<<kCgBlocks, kCgThreads, 0, g.st>>>(xs[i], ys[i], g.n, g.partial + (int64_t)i * kCgBlocks);
  cg_sum_kernel<<<k, kCgThreads, 0, g.st>>>(g.partial, kCgBlocks, g.scal);
  CG_CK(cudaMemcpyAsync(host, g.scal, (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, g.st), "inner products");
  CG_CK(cudaStreamSynchronize(g.st), "inner products");
  return FTOEP_OK;
}

bool is_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

}  // namespace ftoep

using namespace ftoep;

extern "C" ftoep_status ftoep_two_sided_cg(double gamma, double T, int64_t N, const double* f, double* u, double tol,
                                           int maxit, int* iters, double* relres, void* cuda_stream) {
  if (!(gamma > 0.0 && gamma < 1.0) || N < 2 || !(T > 0.0) || !std::isfinite(T) || !(tol > 0.0) || maxit < 1 ||
      !f || !u || N > ((int64_t)1 << 24)) {
    set_global_error("ftoep_two_sided_cg: need 0 < gamma < 1, 2 <= N <= 2^24, T > 0, tol > 0, maxit >= 1, f and u");
    return FTOEP_EINVAL;
  }
  {
    const cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
      char buf[256];
      snprintf(buf, sizeof(buf), "ftoep_two_sided_cg: a CUDA error is pending from earlier work: %s",
               cudaGetErrorString(e));
      set_global_error(buf);
      return FTOEP_ECUDA;
    }
  }
  Cg g;
  g.st = (cudaStream_t)cuda_stream;
  g.n = N - 1;
  g.L = 2;
  while (g.L < 2 * g.n) g.L <<= 1;
  while ((int64_t(1) << g.logL) < g.L) ++g.logL;
  const int64_t n = g.n, L = g.L;
  // first column of A (the L1 weights of weights.cpp: a_0 = mu, a_j = mu (G_j - G_{j-1}))
  std::vector<double> a(n), c(L, 0.0);
  scheme_weights(0, gamma, T / (double)N, n, a.data(), nullptr);
  c[0] = 1.0 + 2.0 * a[0];
  for (int64_t d = 1; d < n; ++d) {
    c[d] = a[d];
    c[L - d] = a[d];
  }
  std::vector<double2> h64;
  host_twiddles(std::max<int64_t>(L, 2), &h64, nullptr, nullptr);
  CG_TRY(g.alloc(&g.c, L * sizeof(double)));
  CG_TRY(g.alloc(&g.tw, h64.size() * sizeof(double2)));
  CG_TRY(g.alloc(&g.spec, L * sizeof(double2)));
  CG_TRY(g.alloc(&g.z, (L / 2) * sizeof(double2)));
  CG_TRY(g.alloc(&g.scratch, L * sizeof(double2)));
  CG_TRY(g.alloc(&g.f, n * sizeof(double)));
  CG_TRY(g.alloc(&g.u, n * sizeof(double)));
  CG_TRY(g.alloc(&g.r, n * sizeof(double)));
  CG_TRY(g.alloc(&g.w, n * sizeof(double)));
  CG_TRY(g.alloc(&g.q, n * sizeof(double)));
  CG_TRY(g.alloc(&g.partial, 2 * kCgBlocks * sizeof(double)));
  CG_TRY(g.alloc(&g.scal, 2 * sizeof(double)));
  CG_CK(cudaMemcpyAsync(g.c, c.data(), L * sizeof(double), cudaMemcpyHostToDevice, g.st), "upload");
  CG_CK(cudaMemcpyAsync(g.tw, h64.data(), h64.size() * sizeof(double2), cudaMemcpyHostToDevice, g.st), "upload");
  CG_CK(cudaMemcpyAsync(g.f, f, n * sizeof(double), is_device(f) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        g.st), "upload");
  CG_CK(cudaMemcpyAsync(g.u, u, n * sizeof(double), is_device(u) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        g.st), "upload");
  SpecArgs sa{};
  sa.a = g.c;
  sa.lo = 0;
  sa.hi = L;
  sa.logn = g.logL;
  sa.nsmem = nsmem_for(P64);
  sa.out = g.spec;
  sa.tw64 = g.tw;
  sa.scratch64 = g.scratch;
  launch_spectrum(P64, sa, g.st);
  if (cudaPeekAtLastError() != cudaSuccess) return cuda_fail("spectrum launch");
  const int eb = (int)std::min<int64_t>(1024, (n + kCgThreads - 1) / kCgThreads);
  // r = f - A u, w = r
  CG_TRY(apply(g, g.u, g.q));
  cg_sub_kernel<<<eb, kCgThreads, 0, g.st>>>(g.r, g.f, g.q, n);
  CG_CK(cudaMemcpyAsync(g.w, g.r, n * sizeof(double), cudaMemcpyDeviceToDevice, g.st), "copy");
  double s2[2];
  {
    const double* xs[2] = {g.r, g.f};
    CG_TRY(dots(g, xs, xs, 2, s2));
  }
  double rr = s2[0];
  const double fnorm = std::sqrt(s2[1]);
  int k = 0;
  while (k < maxit && std::sqrt(rr) > tol * fnorm) {
    CG_TRY(apply(g, g.w, g.q));
    double wq;
    {
      const double* xs[1] = {g.w};
      const double* ys[1] = {g.q};
      CG_TRY(dots(g, xs, ys, 1, &wq));
    }
    if (!(wq > 0.0)) break;  // exact solution reached (or breakdown)
    const double alpha = rr / wq;
    cg_step_kernel<<<eb, kCgThreads, 0, g.st>>>(g.u, g.r, g.w, g.q, alpha, n);
    double rr_new;
    {
      const double* xs[1] = {g.r};
      CG_TRY(dots(g, xs, xs, 1, &rr_new));
    }
    ++k;
    const double beta = rr_new / rr;
    rr = rr_new;
    if (std::sqrt(rr) <= tol * fnorm) break;
    cg_direction_kernel<<<eb, kCgThreads, 0, g.st>>>(g.w, g.r, beta, n);
  }
  // true residual of the result
  CG_TRY(apply(g, g.u, g.q));
  cg_sub_kernel<<<eb, kCgThreads, 0, g.st>>>(g.r, g.f, g.q, n);
  {
    const double* xs[1] = {g.r};
    CG_TRY(dots(g, xs, xs, 1, &rr));
  }
  CG_CK(cudaMemcpyAsync(u, g.u, n * sizeof(double), is_device(u) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        g.st), "download");
  CG_CK(cudaStreamSynchronize(g.st), "download");
  if (iters) *iters = k;
  if (relres) *relres = fnorm > 0.0 ? std::sqrt(rr) / fnorm : std::sqrt(rr);
  return FTOEP_OK;
}
