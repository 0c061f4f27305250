// ftoep_matvec_noalloc: the lower-triangular Toeplitz product y = T x (or T^T x) of
// ftoep_matvec, for callers that must not allocate device memory.
//
// Who needs it: code that runs after its device-memory budget is frozen (a host
// framework whose caching allocator owns the whole device), plugins that the host
// process forbids to allocate, and latency-critical loops where cudaMalloc/cudaFree
// are not acceptable because they can block and synchronise the device.  Such callers
// cannot create a plan (ftoep_create allocates its workspace), so this entry point takes
// only caller-owned inputs and outputs and keeps every intermediate in one static
// device array compiled into the library.
//
// The static array (kNoAllocElems double2 = 16.8 MB) is reserved on every GPU that loads
// the library and held until the process exits.  It is carved into: a pair buffer for
// kNoAllocPairs line pairs, the four-step convolution scratch for those pairs, the kernel
// spectrum, the spectrum scratch and the twiddle tables.  Every call reuses the same
// array: the kernels below rewrite every element they later read (the packing kernel
// writes the zero padding itself), so stale contents from an earlier call never leak into
// a result, but two calls whose GPU work overlaps in time (different streams, or other
// threads) race on the array and must not be issued.
//
// Set-up: on the first call on a device (with that device current) the array's device
// address is looked up with cudaGetSymbolAddress and the twiddle tables are written by a
// kernel; the first call on each device should therefore come before any stream
// capture.  No cudaMalloc, cudaFree or allocating library routine is called, ever.
// The cached address and the twiddle tables belong to the device's context as it was at
// set-up: a device reset (cudaDeviceReset) destroys both and is not supported while the
// library is loaded.
#include <cstdio>
#include <mutex>

#include "../../include/ftoep.h"
#include "internal.h"

using namespace ftoep;

namespace {

constexpr int64_t kNoAllocMaxN = 32768;               // longest line
constexpr int64_t kNoAllocMaxNp = 32768;              // padded line length
constexpr int64_t kNoAllocFFT = 2 * kNoAllocMaxNp;    // longest circulant (65536)
constexpr int64_t kNoAllocPairs = 8;                  // line pairs per batch (16 lines)
constexpr int64_t kOffPairs = 0;
constexpr int64_t kOffScratch = kOffPairs + kNoAllocPairs * kNoAllocMaxNp;
constexpr int64_t kOffSpec = kOffScratch + kNoAllocPairs * kNoAllocFFT;
constexpr int64_t kOffSpecScratch = kOffSpec + kNoAllocFFT;
constexpr int64_t kOffTw = kOffSpecScratch + kNoAllocFFT;
constexpr int64_t kNoAllocElems = kOffTw + 2 * kNoAllocFFT;  // twiddles: 2*nmax - 2 used

static __device__ __align__(256) double2 g_noalloc_scratch[kNoAllocElems];

// W_n^k = exp(-2 pi i k / n) for n = 2 .. kNoAllocFFT at offset n-2 (layout of fft.cuh).
__global__ void noalloc_twiddles(double2* tw) {
  const int64_t tot = 2 * kNoAllocFFT - 2;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t n = 2;
    while (e >= 2 * n - 2) n <<= 1;  // table n covers [n-2, 2n-2)
    const int64_t k = e - (n - 2);
    double s, c;
    sincospi(-2.0 * (double)k / (double)n, &s, &c);
    tw[e] = make_double2(c, s);
  }
}

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double2* g_base[kMaxDevices] = {};

ftoep_status noalloc_setup(double2** base) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    set_global_error("ftoep_matvec_noalloc: no usable current CUDA device");
    return FTOEP_ECUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_base[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      cudaGetLastError();
      set_global_error("ftoep_matvec_noalloc: cudaGetSymbolAddress of the static scratch failed");
      return FTOEP_ECUDA;
    }
    double2* b = (double2*)ptr;
    noalloc_twiddles<<<256, 256>>>(b + kOffTw);
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_global_error("ftoep_matvec_noalloc: twiddle set-up failed");
      return FTOEP_ECUDA;
    }
    g_base[dev] = b;
  }
  *base = g_base[dev];
  return FTOEP_OK;
}

// Device (or managed) memory: the kernels dereference the pointers directly.  Host
// memory, pinned or not, is refused: this entry point stages nothing.
bool on_device(const void* ptr) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();  // the query's own error (unknown pointer), not a pending one
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

ftoep_status launch_failed(const char* step) {
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return FTOEP_OK;
  char buf[256];
  snprintf(buf, sizeof(buf), "ftoep_matvec_noalloc: %s launch failed: %s", step, cudaGetErrorString(e));
  set_global_error(buf);
  return FTOEP_ECUDA;
}

}  // namespace

extern "C" ftoep_status ftoep_matvec_noalloc(const double* a, int64_t N, const double* x, double* y,
                                             int64_t nlines, int transpose, void* cuda_stream) {
  if (!a || !x || !y) {
    set_global_error("ftoep_matvec_noalloc: a, x and y must not be NULL");
    return FTOEP_EINVAL;
  }
  if (N < 1 || N > kNoAllocMaxN) {
    set_global_error("ftoep_matvec_noalloc: N must be in [1, 32768] (size of the static scratch)");
    return FTOEP_EINVAL;
  }
  if (nlines < 1) {
    set_global_error("ftoep_matvec_noalloc: nlines must be >= 1");
    return FTOEP_EINVAL;
  }
  const size_t bytes = (size_t)nlines * (size_t)N * sizeof(double);
  if ((const char*)x < (const char*)y + bytes && (const char*)y < (const char*)x + bytes) {
    set_global_error("ftoep_matvec_noalloc: x and y overlap");
    return FTOEP_EINVAL;
  }
  {  // an error left by earlier work is the caller's: report it without clearing it
    const cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
      char buf[256];
      snprintf(buf, sizeof(buf), "ftoep_matvec_noalloc: a CUDA error is pending from earlier work: %s",
               cudaGetErrorString(e));
      set_global_error(buf);
      return FTOEP_ECUDA;
    }
  }
  if (!on_device(a) || !on_device(x) || !on_device(y)) {
    set_global_error("ftoep_matvec_noalloc: a, x and y must be device (or managed) memory; host buffers go "
                     "through ftoep_matvec");
    return FTOEP_EINVAL;
  }
  double2* base = nullptr;
  ftoep_status s = noalloc_setup(&base);
  if (s != FTOEP_OK) return s;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int64_t Np = 16;
  while (Np < N) Np <<= 1;
  int logn = 0;
  while ((int64_t(1) << logn) < 2 * Np) ++logn;

  SpecArgs sa{};
  sa.a = a;
  sa.lo = 0;
  sa.hi = N;
  sa.logn = logn;
  sa.nsmem = nsmem_for(P64);
  sa.out = base + kOffSpec;
  sa.tw64 = base + kOffTw;
  sa.scratch64 = base + kOffSpecScratch;
  launch_spectrum(P64, sa, st);
  if ((s = launch_failed("kernel spectrum")) != FTOEP_OK) return s;
  for (int64_t l0 = 0; l0 < nlines; l0 += 2 * kNoAllocPairs) {
    const int64_t nl = (nlines - l0 < 2 * kNoAllocPairs) ? nlines - l0 : 2 * kNoAllocPairs;
    PackArgs pa{};
    pa.x = x + l0 * N;
    pa.y = y + l0 * N;
    pa.z = base + kOffPairs;
    pa.ld = Np;
    pa.N = N;
    pa.nlines = nl;
    pa.reverse = transpose ? 1 : 0;
    pa.mode = 0;
    launch_pack(P64, pa, st);
    if ((s = launch_failed("packing")) != FTOEP_OK) return s;
    ConvArgs ca{};
    ca.zin = base + kOffPairs;
    ca.zout = base + kOffPairs;
    ca.ld_in = ca.ld_out = Np;
    ca.in_off = ca.out_off = 0;
    ca.npairs = (nl + 1) / 2;
    ca.logn = logn;
    ca.nsmem = nsmem_for(P64);
    ca.mode = 1;
    ca.spec = base + kOffSpec;
    ca.tw = base + kOffTw;
    ca.scratch = base + kOffScratch;
    launch_conv(P64, ca, st);
    if ((s = launch_failed("circulant convolution")) != FTOEP_OK) return s;
    launch_unpack(P64, pa, st);
    if ((s = launch_failed("unpacking")) != FTOEP_OK) return s;
  }
  return FTOEP_OK;
}
