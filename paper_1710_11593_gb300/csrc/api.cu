// C ABI of libftoep (include/ftoep.h): plans, workspaces, streams and the order of the
// kernels.
//
// ftoep_solve, per problem (difference form, see solve_problem):
//   1. right-hand side + sine transform along space      -> mode pairs z[P][Np]
//   2. per time block of length B: the block solve as a causal convolution with the
//      per-mode block inverse; then the one cross-block update that becomes due (level
//      s = B * 2^ctz(block+1)) as a circulant convolution
//   3. inverse sine transform, u = u0 + tau * cumsum(v)
//   mixed precision: 1-3 in float (running sums of the all-ones part in double), then the
//   residual of the same difference-form rows (float-float Toeplitz product, spatial
//   stencil in double), 1-3 on it, u += correction.
// A plan with several problems runs them on internal streams (4 unless tuned; longest
// first, each onto the least-loaded stream), each stream with its own workspace; the
// caller's stream forks to them and joins them again through events.  Device-pointer
// solves are captured once as a CUDA graph and replayed (solve_device).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ftoep.h"
#include "internal.h"

using namespace ftoep;

namespace {

constexpr int kMaxStreams = 8;
constexpr int kDefaultStreams = 4;
constexpr int kNumClasses = 8;
constexpr int kDotBlocks = 1024;

struct Prob {
  ftoep_problem d{};
  int tk = 0;                   // family of the time weights: 0 (L1, Eq. 4/19) or 1 (Eq. 15/17)
  double sw = 1.0;              // share of the spatial operator on the level-n diagonal (1/2: Crank-Nicolson)
  int64_t N = 0, M = 0, Np = 0, P = 0;
  int logNp = 0, logK2 = 0;
  double tau = 0, h = 0, scale = 0;
  int B = 0, L = 0, Sf = 0, nblk = 0;
  int64_t ncols = 0;
  Prec prec = P64;
  int64_t foff = 0, voff = 0;
  int stream = 0;               // internal stream the problem runs on
  double cost = 0;              // scheduling estimate
  double pair_cost = 0;         // one pair's chain (block solves and cross-block levels)
  int group = -1;               // chain schedule: group of the problem
  size_t zbyte = 0;             // chain schedule: offset of its pair array in the group buffer
  std::vector<double> h_a, h_dadg;
  double* a = nullptr;          // first column of the time operator (original form)
  double* dadg = nullptr;       // its derivative in gamma
  double* e = nullptr;          // first column in the difference form (solve kernel)
  double* wu0 = nullptr;
  double* wphi = nullptr;
  double2* invdiag = nullptr;   // per pair 1/(e_0 + sw lambda tau)
  double2* lamtau = nullptr;    // per pair lambda tau
  // sine transform for M+1 not a power of two (Bluestein tables, double and float)
  bool bluestein = false;
  double2* chirp64 = nullptr;
  double2* bspec64 = nullptr;
  float2* chirp32 = nullptr;
  float2* bspec32 = nullptr;
  double* sinv64 = nullptr;     // sin(pi j/K), j <= K/2 (double, folded form)
  int logP64 = 0, logP32 = 0;   // chirp-z lengths of the double (folded) and float (odd) forms
  void* spec = nullptr;         // solve spectra, precision prec
  double2* spec64 = nullptr;    // solve spectra in double (adjoint of mixed problems; == spec for P64)
  double2* spec_mv = nullptr;   // product spectrum, length 2Np
  double2* spec_dg = nullptr;   // d/dgamma product spectrum
  void* spec_res = nullptr;     // float-float spectrum of the difference-form kernel (mixed residual)
  // block inverse spectra (block_inverse.cu): precision of the solve, and double (adjoint)
  void* c1 = nullptr;
  void* c2 = nullptr;
  // inverse-series solve: packed spectra of the whole inverse columns [P][2Np] (solve precision)
  bool finv = false;
  void* cinv = nullptr;
  double2* c1_64 = nullptr;
  double2* c2_64 = nullptr;
};

// One stream's workspace.
struct Ws {
  cudaStream_t st = nullptr;
  bool own = false;
  void* z = nullptr;             // solve pairs (max P*Np double2)
  void* scratch = nullptr;       // four-step scratch of the solve (max P*Np double2)
  double2* zmv = nullptr;        // product pairs (max P*Np double2)
  double2* scratch_mv = nullptr; // four-step scratch of products (max P*2Np double2)
  double* r = nullptr;           // residual / temporary field (max M*N)
  double2* prefix = nullptr;     // running sums of the difference-form solve (max P)
  double* dpart = nullptr;       // reduction partials
  // host-pointer staging (per problem, allocated on first use)
  double* stage_in = nullptr;
  double* stage_out = nullptr;
  double* stage_v0 = nullptr;
  double* stage_v1 = nullptr;
  double* stage_u = nullptr;
  cudaEvent_t done = nullptr;
};

int ilog2(int64_t v) {
  int l = 0;
  while ((int64_t(1) << l) < v) ++l;
  return l;
}
bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
int ctz64(int64_t v) {
  int c = 0;
  while (!(v & 1)) {
    v >>= 1;
    ++c;
  }
  return c;
}

thread_local std::string g_create_error;

}  // namespace

namespace ftoep {
// Message for ftoep_last_error(NULL, ...) from entry points that have no plan.
void set_global_error(const char* msg) { g_create_error = msg; }

// Twiddle tables W_n^k = exp(-2 pi i k/n) for every power of two n = 2 .. maxtw at offset
// n-2 (layout of fft.cuh), in double, float and float-float, from one long-double table.
void host_twiddles(int64_t maxtw, std::vector<double2>* h64, std::vector<float2>* h32, std::vector<float4>* hff) {
  const size_t tot = (size_t)2 * maxtw - 2;
  if (h64) h64->resize(tot);
  if (h32) h32->resize(tot);
  if (hff) hff->resize(tot);
  std::vector<double2> big(maxtw);
  std::vector<float4> bigff(maxtw);
  const long double two_pi = 6.283185307179586476925286766559005768L;
  for (int64_t k = 0; k < maxtw; ++k) {
    long double ang = -two_pi * (long double)k / (long double)maxtw;
    const long double c = cosl(ang), sn = sinl(ang);
    big[k] = make_double2((double)c, (double)sn);
    const float ch = (float)c, sh = (float)sn;
    bigff[k] = make_float4(ch, (float)(c - (long double)ch), sh, (float)(sn - (long double)sh));
  }
  for (int64_t n = 2; n <= maxtw; n <<= 1) {
    const int64_t stride = maxtw / n;
    for (int64_t k = 0; k < n; ++k) {
      if (h64) (*h64)[(n - 2) + k] = big[k * stride];
      if (h32) (*h32)[(n - 2) + k] = make_float2((float)big[k * stride].x, (float)big[k * stride].y);
      if (hff) (*hff)[(n - 2) + k] = bigff[k * stride];
    }
  }
}
}  // namespace ftoep

// A solve captured as a CUDA graph for one set of device pointers (see ftoep_solve).
struct SolveGraph {
  const void* f = nullptr;
  const void* u = nullptr;
  const void* u0 = nullptr;
  const void* phi = nullptr;
  int runs = 0;                   // direct runs seen before the capture
  cudaGraphExec_t exec = nullptr;
  int64_t launches[kNumClasses] = {};  // kernels per replay, per class
};

// Chain schedule: problems whose pair arrays are resident together, solved by one
// persistent launch per precision (chain.cu).
struct ChainGroup {
  std::vector<int> probs;          // problem indices, longest chains first
  ChainProb* d_probs = nullptr;    // device descriptors of its problems
  int2* d_items[2] = {nullptr, nullptr};  // per precision (0 double, 1 float): (descriptor, pair)
  int nitems[2] = {0, 0};
  size_t bytes = 0;                // pair arrays of the group
};

struct ftoep_plan_s {
  std::vector<Prob> probs;
  // Fault injection on the host: with FTOEP_FAIL_ALLOC_AFTER=k in the environment at plan
  // creation, the plan's device allocations fail (FTOEP_ENOMEM) after its first k -- the
  // out-of-memory paths without exhausting a GPU.
  long fail_after = -1;
  long nalloc = 0;
  int sched = 1;                  // 1: per-level launches, 2: persistent per-pair chains
  std::vector<ChainGroup> groups;
  void* gz = nullptr;             // pair arrays of the current group
  unsigned* counters = nullptr;   // one work counter per chain launch of a solve
  int ncounters = 0;
  void* chain_scr[2] = {nullptr, nullptr};
  int64_t chain_scr_el[2] = {0, 0};
  int chain_grid[2] = {0, 0};
  size_t chain_smem[2] = {0, 0};
  cudaStream_t stream = nullptr;  // caller's stream
  int device = 0;
  int64_t ntw = 0;
  double2* tw64 = nullptr;
  float2* tw32 = nullptr;
  void* twff = nullptr;           // float-float twiddles (ff2)
  std::vector<Ws> ws;
  size_t z_el = 0, mv_el = 0, r_el = 0, p_el = 0, v_el = 0;
  size_t scr_el = 0;  // solve scratch (double2): the largest P*Np, and 2 Np of an inverse-series problem
  double* dscal = nullptr;        // device scalars (nprob)
  cudaEvent_t fork = nullptr;
  int64_t total_field = 0, total_vec = 0;
  std::string err;
  std::vector<void*> allocs;
  // launch counters (always on) and optional CUDA-event timing per kernel class
  bool prof_on = false;
  int64_t launches[kNumClasses] = {};
  double prof_ms[kNumClasses] = {};
  int64_t prof_ops[kNumClasses] = {};
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  std::vector<cudaEvent_t> evpool;
  std::vector<SolveGraph> graphs;  // most recently used last
  cudaStream_t gstream = nullptr;  // root stream the graphs are captured and replayed on
  cudaEvent_t gev_in = nullptr, gev_out = nullptr;
  // host-buffer solves on the chain schedule: device copies of one group's f and u (when
  // they fit), so that f crosses the host link once and u once per solve
  double* res_f = nullptr;
  double* res_u = nullptr;
  bool res_tried = false;
};

namespace {

ftoep_status fail(ftoep_plan p, ftoep_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (p) p->err = buf; else g_create_error = buf;
  return s;
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail(pl, e_ == cudaErrorMemoryAllocation ? FTOEP_ENOMEM : FTOEP_ECUDA,   \
                  "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

#define CKL()                                                                         \
  do {                                                                                \
    cudaError_t e_ = cudaGetLastError();                                              \
    if (e_ != cudaSuccess)                                                            \
      return fail(pl, FTOEP_ECUDA, "kernel launch: %s (%s:%d)", cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

ftoep_status dalloc(ftoep_plan pl, void** out, size_t bytes) {
  *out = nullptr;
  if (bytes == 0) return FTOEP_OK;
  if (pl->fail_after >= 0 && pl->nalloc++ >= pl->fail_after)
    return fail(pl, FTOEP_ENOMEM, "cudaMalloc(%zu bytes): refused by FTOEP_FAIL_ALLOC_AFTER", bytes);
  cudaError_t e = cudaMalloc(out, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *out = nullptr;
    return fail(pl, FTOEP_ENOMEM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
  }
  pl->allocs.push_back(*out);
  return FTOEP_OK;
}

cudaEvent_t ev_get(ftoep_plan pl) {
  if (!pl->evpool.empty()) {
    cudaEvent_t e = pl->evpool.back();
    pl->evpool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Launch on stream `st` (in scope) through a launcher that returns its kernel count;
// count it, optionally time it with a pair of events on the same stream.
#define LAUNCH(cls, expr)                                            \
  do {                                                               \
    cudaEvent_t e0_ = nullptr, e1_ = nullptr;                        \
    if (pl->prof_on) {                                               \
      e0_ = ev_get(pl);                                              \
      e1_ = ev_get(pl);                                              \
      cudaEventRecord(e0_, st);                                      \
    }                                                                \
    pl->launches[(cls)] += (expr);                                   \
    if (pl->prof_on) {                                               \
      cudaEventRecord(e1_, st);                                      \
      pl->pending.push_back({(cls), {e0_, e1_}});                    \
    }                                                                \
    CKL();                                                           \
  } while (0)

#define ALLOC(ptr, bytes)                                                  \
  do {                                                                     \
    ftoep_status s_ = dalloc(pl, (void**)&(ptr), (bytes));                 \
    if (s_ != FTOEP_OK) return s_;                                         \
  } while (0)

#define TRY(expr)                          \
  do {                                     \
    ftoep_status s_ = (expr);              \
    if (s_ != FTOEP_OK) return s_;         \
  } while (0)

bool is_device_ptr(const void* ptr) {
  if (!ptr) return true;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

const void* tw_of(ftoep_plan pl, Prec pr) {
  return pr == P64 ? (const void*)pl->tw64 : pr == P32 ? (const void*)pl->tw32 : (const void*)pl->twff;
}
size_t velem(Prec pr) { return pr == P32 ? sizeof(float2) : sizeof(double2); }

void release(ftoep_plan pl, void* ptr) {
  if (!ptr) return;
  for (auto it = pl->allocs.begin(); it != pl->allocs.end(); ++it) {
    if (*it == ptr) {
      cudaFree(ptr);
      pl->allocs.erase(it);
      return;
    }
  }
}

ftoep_status validate(const ftoep_problem& d, int i, const ftoep_tuning* tune) {
  ftoep_plan pl = nullptr;
  if (d.kind == FTOEP_L1_SUBDIFFUSION) {
    if (!(d.gamma > 0.0 && d.gamma < 1.0)) return fail(pl, FTOEP_EINVAL, "problem %d: gamma %g not in (0,1)", i, d.gamma);
  } else if (d.kind == FTOEP_L1_HYPERBOLIC || d.kind == FTOEP_L1_HYPERBOLIC_CN) {
    if (!(d.gamma > 1.0 && d.gamma < 2.0)) return fail(pl, FTOEP_EINVAL, "problem %d: gamma %g not in (1,2)", i, d.gamma);
  } else {
    return fail(pl, FTOEP_EINVAL, "problem %d: unknown kind %d", i, d.kind);
  }
  if (d.space != FTOEP_SPACE_NONE && d.space != FTOEP_SPACE_DIRICHLET_LAPLACIAN)
    return fail(pl, FTOEP_EINVAL, "problem %d: unknown space %d", i, d.space);
  if (d.precision != FTOEP_FP64 && d.precision != FTOEP_MIXED)
    return fail(pl, FTOEP_EINVAL, "problem %d: unknown precision %d", i, d.precision);
  if (d.N < 1 || d.M < 1) return fail(pl, FTOEP_EINVAL, "problem %d: N=%lld M=%lld must be >= 1", i, (long long)d.N, (long long)d.M);
  if (!(d.T > 0.0) || !std::isfinite(d.T)) return fail(pl, FTOEP_EINVAL, "problem %d: T must be > 0", i);
  if (d.space == FTOEP_SPACE_DIRICHLET_LAPLACIAN && (!(d.L > 0.0) || !std::isfinite(d.L)))
    return fail(pl, FTOEP_EINVAL, "problem %d: L must be > 0", i);
  if (d.space == FTOEP_SPACE_NONE && (!(d.lambda >= 0.0) || !std::isfinite(d.lambda)))
    return fail(pl, FTOEP_EINVAL, "problem %d: lambda must be >= 0", i);
  if (d.N > (int64_t(1) << 22)) return fail(pl, FTOEP_EUNSUPPORTED, "problem %d: N > 2^22 not supported", i);
  if (d.space == FTOEP_SPACE_DIRICHLET_LAPLACIAN) {
    const Prec pr = d.precision == FTOEP_FP64 ? P64 : P32;
    const int64_t lim = is_pow2(d.M + 1) ? (d.precision == FTOEP_FP64 ? 4096 : 8192) : bluestein_max_K(pr);
    if (d.M + 1 > lim) return fail(pl, FTOEP_EUNSUPPORTED, "problem %d: M+1 = %lld > %lld not supported", i,
                                   (long long)(d.M + 1), (long long)lim);
  }
  if (tune) {
    if (tune->leaf && (!is_pow2(tune->leaf) || tune->leaf > 16))
      return fail(pl, FTOEP_EINVAL, "tuning: leaf must be a power of two <= 16");
    if (tune->fft_tile && (!is_pow2(tune->fft_tile) || tune->fft_tile > 4096 || tune->fft_tile < 16))
      return fail(pl, FTOEP_EINVAL, "tuning: fft_tile must be a power of two in [16, 4096]");
    if (tune->gemm_max_level && (!is_pow2(tune->gemm_max_level) || tune->gemm_max_level > 2048))
      return fail(pl, FTOEP_EINVAL, "tuning: gemm_max_level must be a power of two <= 2048");
    if (tune->streams < 0 || tune->streams > kMaxStreams)
      return fail(pl, FTOEP_EINVAL, "tuning: streams must be in [0, %d]", kMaxStreams);
    if (tune->solver < 0 || tune->solver > FTOEP_SOLVER_INVERSE_MIXED_SUBDIFFUSION)
      return fail(pl, FTOEP_EINVAL, "tuning: solver %d unknown", tune->solver);
    if (tune->scheduler < 0 || tune->scheduler > FTOEP_SCHED_CHAIN)
      return fail(pl, FTOEP_EINVAL, "tuning: scheduler must be 0 (library choice), 1 (levels) or 2 (chain)");
  }
  return FTOEP_OK;
}

// Spectra of the solve levels s = Sf .. Np/2 (level s at offset 2(s - Sf)).
ftoep_status build_solve_spectra(ftoep_plan pl, Ws& w, Prob& pb, Prec pr, void* out) {
  cudaStream_t st = w.st;
  for (int64_t s = pb.Sf; s <= pb.Np / 2; s <<= 1) {
    SpecArgs sa{};
    sa.a = pb.e;
    sa.lo = 1;
    sa.hi = 2 * s;
    sa.logn = ilog2(2 * s);
    sa.nsmem = nsmem_for(pr);
    sa.out = (char*)out + (size_t)2 * (s - pb.Sf) * velem(pr);
    sa.tw64 = pl->tw64;
    sa.scratch64 = w.scratch_mv;
    LAUNCH(FTOEP_K_OTHER, launch_spectrum(pr, sa, st));
  }
  return FTOEP_OK;
}

// Spectrum of the full product y = T x (c_k = coeff_k for k < N, zero after), length
// 2Np, in precision pr (double or float-float).
ftoep_status build_product_spectrum(ftoep_plan pl, Ws& w, Prob& pb, const double* coeff, void** out, Prec pr) {
  if (*out) return FTOEP_OK;
  cudaStream_t st = w.st;
  ALLOC(*out, (size_t)2 * pb.Np * velem(pr));
  SpecArgs sa{};
  sa.a = coeff;
  sa.lo = 0;
  sa.hi = pb.N;
  sa.logn = pb.logNp + 1;
  sa.nsmem = nsmem_for(pr);
  sa.out = *out;
  sa.tw64 = pl->tw64;
  sa.scratch64 = w.scratch_mv;
  LAUNCH(FTOEP_K_OTHER, launch_spectrum(pr, sa, st));
  return FTOEP_OK;
}

// In-place difference-form solve of the pair array z (right-hand side in, v out).
ftoep_status solve_pairs(ftoep_plan pl, Ws& w, Prob& pb, Prec pr, void* z, const void* spec) {
  cudaStream_t st = w.st;
  if (pb.finv && pr == pb.prec) {  // inverse-series solve: one convolution of length 2 Np per pair
    // pairs in chunks whose scratch (2 Np values each) fits the stream's scratch
    const int64_t n = 2 * pb.Np;
    const int64_t chunk = std::max<int64_t>(1, (int64_t)(pl->scr_el * sizeof(double2) / ((size_t)n * velem(pr))));
    for (int64_t p0 = 0; p0 < pb.P; p0 += chunk) {
      FinvArgs fa{};
      fa.z = (char*)z + (size_t)p0 * pb.Np * velem(pr);
      fa.ld = pb.Np;
      fa.N = pb.N;
      fa.npairs = std::min<int64_t>(chunk, pb.P - p0);
      fa.logn = pb.logNp + 1;
      fa.cs = (const char*)pb.cinv + (size_t)p0 * n * velem(pr);
      fa.tw = tw_of(pl, pr);
      fa.scratch = w.scratch;
      LAUNCH(FTOEP_K_INVERSE, launch_full_inverse(pr, fa, st));
    }
    return FTOEP_OK;
  }
  CK(cudaMemsetAsync(w.prefix, 0, (size_t)pb.P * sizeof(double2), st));
  const void* c1 = pr == pb.prec ? pb.c1 : (const void*)pb.c1_64;
  const void* c2 = pr == pb.prec ? pb.c2 : (const void*)pb.c2_64;
  for (int b = 0; b < pb.nblk; ++b) {
    BlockInvArgs bi{};
    bi.z = z;
    bi.ld = pb.Np;
    bi.npairs = pb.P;
    bi.t0 = (int64_t)b * pb.B;
    bi.B = pb.B;
    bi.logB = ilog2(pb.B);
    bi.c1 = c1;
    bi.c2 = c2;
    bi.lamtau = pb.lamtau;
    bi.prefix = w.prefix;
    bi.tw = tw_of(pl, pr);
    LAUNCH(FTOEP_K_BLOCK_SOLVE, launch_block_inverse(pr, bi, st));
    const int64_t v = b + 1;
    if (v < pb.nblk) {
      const int64_t s = (int64_t)pb.B << ctz64(v);
      const int64_t mid = v * pb.B;
      ConvArgs ca{};
      ca.zin = z;
      ca.zout = z;
      ca.ld_in = ca.ld_out = pb.Np;
      ca.in_off = mid - s;
      ca.out_off = mid;
      ca.npairs = pb.P;
      ca.logn = ilog2(2 * s);
      ca.nsmem = nsmem_for(pr);
      ca.mode = 0;
      ca.spec = (const char*)spec + (size_t)2 * (s - pb.Sf) * velem(pr);
      ca.tw = tw_of(pl, pr);
      ca.scratch = w.scratch;
      LAUNCH((2 * s <= nsmem_for(pr)) ? FTOEP_K_CONV_SMEM : FTOEP_K_CONV_FOURSTEP, launch_conv(pr, ca, st));
    }
  }
  return FTOEP_OK;
}

DstArgs dst_args(ftoep_plan pl, const Prob& pb, Prec pr, void* z) {
  DstArgs da{};
  da.z = z;
  da.ld = pb.Np;
  da.N = pb.N;
  da.ncols = pb.ncols;
  da.M = pb.M;
  da.logK2 = pb.logK2;
  da.space = pb.d.space;
  da.inv_h2 = 1.0 / (pb.h * pb.h);
  da.lambda = pb.d.lambda;
  da.tw = tw_of(pl, pr);
  da.dst_scale = 1.0 / std::sqrt(2.0 * (double)(pb.M + 1));
  if (pb.bluestein) {
    da.bluestein = 1;
    da.K = (int)(pb.M + 1);
    da.chirp = pr == P64 ? (const void*)pb.chirp64 : (const void*)pb.chirp32;
    da.bspec = pr == P64 ? (const void*)pb.bspec64 : (const void*)pb.bspec32;
    da.sinv = pr == P64 ? (const void*)pb.sinv64 : nullptr;
    da.logP = pr == P64 ? pb.logP64 : pb.logP32;
  }
  return da;
}

// y = T x on nlines lines of length N (double in and out, arithmetic in precision pr:
// double or float-float), through the product workspace.  cls >= 0 books every launch
// under that kernel class instead of the transform/convolution classes.
ftoep_status product_lines(ftoep_plan pl, Ws& w, Prob& pb, Prec pr, const void* spec, const double* x,
                           double* y_or_null, int64_t nlines, int reverse, int cls = -1, const float* x32 = nullptr) {
  cudaStream_t st = w.st;
  PackArgs pa{};
  pa.x = x;
  pa.x32 = x32;
  pa.z = w.zmv;
  pa.ld = pb.Np;
  pa.N = pb.N;
  pa.nlines = nlines;
  pa.reverse = reverse;
  LAUNCH(cls >= 0 ? cls : FTOEP_K_OTHER, launch_pack(pr, pa, st));
  ConvArgs ca{};
  ca.zin = w.zmv;
  ca.zout = w.zmv;
  ca.ld_in = ca.ld_out = pb.Np;
  ca.in_off = ca.out_off = 0;
  ca.npairs = (nlines + 1) / 2;
  ca.logn = pb.logNp + 1;
  ca.nsmem = nsmem_for(pr);
  ca.mode = 1;
  ca.spec = spec;
  ca.tw = tw_of(pl, pr);
  ca.scratch = w.scratch_mv;
  LAUNCH(cls >= 0 ? cls : (2 * pb.Np <= nsmem_for(pr)) ? FTOEP_K_CONV_SMEM : FTOEP_K_CONV_FOURSTEP,
         launch_conv(pr, ca, st));
  if (y_or_null) {
    pa.y = y_or_null;
    pa.mode = 0;
    LAUNCH(cls >= 0 ? cls : FTOEP_K_OTHER, launch_unpack(pr, pa, st));
  }
  return FTOEP_OK;
}

// Time sums along every line: u = base + tau * cumsum(in) (or tau * suffix sums); in32:
// float input (forward only).
ftoep_status scan_lines(ftoep_plan pl, Ws& w, Prob& pb, const double* in, double* out, const double* u0, int accumulate,
                        int reverse, const float* in32 = nullptr) {
  cudaStream_t st = w.st;
  ScanArgs sc{};
  sc.in = in;
  sc.in32 = in32;
  sc.tau_h = (float)pb.tau;
  sc.tau_l = (float)(pb.tau - (double)sc.tau_h);
  sc.out = out;
  sc.u0 = u0;
  sc.N = pb.N;
  sc.M = pb.M;
  sc.tau = pb.tau;
  sc.accumulate = accumulate;
  sc.reverse = reverse;
  LAUNCH(FTOEP_K_OTHER, launch_scan(sc, st));
  return FTOEP_OK;
}

// The solve runs on the difference quotients v_n = (u^n - u^{n-1})/tau: per mode the
// operator is E + lambda_m tau 1 (E lower-triangular Toeplitz, shared; 1 the all-ones
// lower triangle) with right-hand side f + [c tau M_{n-1} phi] - S u0, and
// u = u0 + tau cumsum(v).  Written in v the history terms carry the scale tau^(1-g)
// instead of tau^-g, which keeps float arithmetic usable at large N.
//
// A problem's solve in three pieces around its pair solves (per-level launches, or the
// persistent chain over a group of problems):
//   rhs_forward        right-hand side + forward sine transform -> pairs z
//   after_first_solve  inverse transform + time sums -> u; mixed: residual of the same
//                      rows and its forward transform -> z (the correction's right-hand side)
//   after_correction   mixed: inverse transform of the correction, u += tau cumsum

// Right-hand side of the difference form and its forward sine transform into z.
ftoep_status rhs_forward(ftoep_plan pl, Ws& w, Prob& pb, void* z, const double* f, const double* u0,
                         const double* phi) {
  cudaStream_t st = w.st;
  DstArgs da = dst_args(pl, pb, pb.prec, z);
  da.f = f;
  da.u0 = u0;
  da.phi = (pb.tk == 1) ? phi : nullptr;
  da.wu0 = pb.wu0;
  da.wphi = pb.wphi;
  da.diff_form = 1;
  LAUNCH(FTOEP_K_SINE, launch_dst_forward(pb.prec, da, st));
  return FTOEP_OK;
}

// z holds the solved v in mode space.  Double: u = u0 + tau cumsum(S^-1 v).  Mixed: the
// same in float-float time sums, then the residual r = f + c tau M phi - E v - S u of the
// same rows (E v in float-float, f - S u in double) and its forward transform into z.
ftoep_status after_first_solve(ftoep_plan pl, Ws& w, Prob& pb, void* z, const double* f, double* u,
                               const double* u0, const double* phi) {
  cudaStream_t st = w.st;
  const Prec pr = pb.prec;
  DstArgs da = dst_args(pl, pb, pr, z);
  if (pr == P64) {
    da.u = u;
    da.accumulate = 0;
    LAUNCH(FTOEP_K_SINE, launch_dst_inverse(pr, da, st));
    TRY(scan_lines(pl, w, pb, u, u, u0, 0, 0));
    return FTOEP_OK;
  }
  // mixed: the solved v (physical space) in float in r, u = u0 + tau cumsum(v)
  float* r32 = (float*)w.r;
  da.u32 = r32;
  da.accumulate = 0;
  LAUNCH(FTOEP_K_SINE, launch_dst_inverse(pr, da, st));
  TRY(scan_lines(pl, w, pb, nullptr, u, u0, 0, 0, r32));
  // residual of the same rows in the difference form, r = f + c tau M phi - E v - S u,
  // with the Toeplitz product E v in float-float (no tau^-g cancellation in this form)
  TRY(product_lines(pl, w, pb, PFF, pb.spec_res, nullptr, nullptr, pb.M, 0, FTOEP_K_RESIDUAL, r32));
  ResidualArgs ra{};
  ra.f = f;
  ra.u0 = nullptr;
  ra.phi = (pb.tk == 1) ? phi : nullptr;
  ra.cn = pb.sw != 1.0;
  ra.uprev0 = u0;  // Crank-Nicolson: the level before the first is u0 (zero if NULL)
  ra.wu0 = pb.wu0;
  ra.wphi = pb.wphi;
  ra.u = u;
  ra.tu = w.zmv;
  ra.r32 = r32;
  ra.ld = pb.Np;
  ra.N = pb.N;
  ra.M = pb.M;
  ra.space = pb.d.space;
  ra.inv_h2 = 1.0 / (pb.h * pb.h);
  ra.lambda = pb.d.lambda;
  LAUNCH(FTOEP_K_RESIDUAL, launch_residual(ra, st));
  // correction: same rows, zero initial data
  DstArgs dr = dst_args(pl, pb, pr, z);
  dr.f32 = r32;
  dr.diff_form = 1;
  LAUNCH(FTOEP_K_SINE, launch_dst_forward(pr, dr, st));
  return FTOEP_OK;
}

// Mixed: z holds the solved correction; u += tau cumsum(S^-1 z).
ftoep_status after_correction(ftoep_plan pl, Ws& w, Prob& pb, void* z, double* u) {
  cudaStream_t st = w.st;
  float* r32 = (float*)w.r;
  DstArgs dr = dst_args(pl, pb, pb.prec, z);
  dr.u32 = r32;
  dr.accumulate = 0;
  LAUNCH(FTOEP_K_SINE, launch_dst_inverse(pb.prec, dr, st));
  TRY(scan_lines(pl, w, pb, nullptr, u, nullptr, 1, 0, r32));
  return FTOEP_OK;
}

ftoep_status ensure_level_ws(ftoep_plan pl, Ws& w);

// One problem with per-level launches on the stream's own pair array.
ftoep_status solve_problem(ftoep_plan pl, Ws& w, Prob& pb, const double* f, double* u, const double* u0,
                           const double* phi) {
  TRY(ensure_level_ws(pl, w));
  TRY(rhs_forward(pl, w, pb, w.z, f, u0, phi));
  TRY(solve_pairs(pl, w, pb, pb.prec, w.z, pb.spec));
  TRY(after_first_solve(pl, w, pb, w.z, f, u, u0, phi));
  if (pb.prec == P64) return FTOEP_OK;
  TRY(solve_pairs(pl, w, pb, pb.prec, w.z, pb.spec));
  return after_correction(pl, w, pb, w.z, u);
}

// Adjoint of one problem (double): dldf = A_u^-T g and, if dgamma_out, the partial
// <dldf, (dA/dgamma) u> into *dgamma_out (device).
ftoep_status adjoint_problem(ftoep_plan pl, Ws& w, Prob& pb, const double* g, const double* u, double* dldf,
                             double* dgamma_out) {
  cudaStream_t st = w.st;
  if (pb.bluestein && pb.M + 1 > bluestein_max_K(P64))
    return fail(pl, FTOEP_EUNSUPPORTED, "adjoint: M+1 = %lld > %d needs a double sine transform that is not built",
                (long long)(pb.M + 1), bluestein_max_K(P64));
  TRY(ensure_level_ws(pl, w));
  // The adjoint runs in double with the problem's own block length (and the double block
  // inverse spectra: c1/c2 of a mixed problem are float).
  Prob q = pb;
  q.prec = P64;
  q.c1 = pb.c1_64;
  q.c2 = pb.c2_64;
  if (pb.prec != P64) q.finv = false;  // the inverse spectra of a mixed problem are float
  // With u = tau C v (C the all-ones lower triangle), A_u = A_v (tau C)^-1, so
  // A_u^-T g = A_v^-T (tau C^T g): suffix sums of g, then the transposed difference-form
  // solve, done as time reversal + forward solve + reversal (J A_v^T J = A_v per mode).
  TRY(scan_lines(pl, w, pb, g, w.r, nullptr, 0, 1));
  DstArgs da = dst_args(pl, q, P64, w.z);
  da.f = w.r;
  da.reverse = 1;
  LAUNCH(FTOEP_K_SINE, launch_dst_forward(P64, da, st));
  TRY(solve_pairs(pl, w, q, P64, w.z, pb.spec64));
  da.u = dldf;
  da.accumulate = 0;
  LAUNCH(FTOEP_K_SINE, launch_dst_inverse(P64, da, st));
  if (dgamma_out) {
    TRY(product_lines(pl, w, pb, P64, pb.spec_dg, u, nullptr, pb.M, 0));
    DotArgs dt{};
    dt.x = dldf;
    dt.tu = w.zmv;
    dt.ld = pb.Np;
    dt.N = pb.N;
    dt.nlines = pb.M;
    dt.partial = w.dpart;
    dt.nblocks = kDotBlocks;
    LAUNCH(FTOEP_K_OTHER, launch_dot(dt, st));
    LAUNCH(FTOEP_K_OTHER, launch_sum(w.dpart, kDotBlocks, dgamma_out, st));
  }
  return FTOEP_OK;
}

// Pair array and four-step scratch of a stream's per-level solves (allocated on first use
// when the plan runs the chain schedule).
ftoep_status ensure_level_ws(ftoep_plan pl, Ws& w) {
  if (!w.z) {
    ALLOC(w.z, pl->z_el * sizeof(double2));
    CK(cudaMemsetAsync(w.z, 0, pl->z_el * sizeof(double2), w.st));
  }
  if (!w.scratch) ALLOC(w.scratch, pl->scr_el * sizeof(double2));
  return FTOEP_OK;
}

ftoep_status ensure_staging(ftoep_plan pl, Ws& w) {
  if (w.stage_in) return FTOEP_OK;
  ALLOC(w.stage_in, pl->r_el * sizeof(double));
  ALLOC(w.stage_out, pl->r_el * sizeof(double));
  ALLOC(w.stage_u, pl->r_el * sizeof(double));
  ALLOC(w.stage_v0, pl->v_el * sizeof(double));
  ALLOC(w.stage_v1, pl->v_el * sizeof(double));
  return FTOEP_OK;
}

ftoep_status sync_plan(ftoep_plan pl) {
  cudaError_t e = cudaStreamSynchronize(pl->stream);
  if (e != cudaSuccess) return fail(pl, FTOEP_ECUDA, "stream synchronize: %s", cudaGetErrorString(e));
  return FTOEP_OK;
}

// Device copies of the fields of the largest chain group, for host-buffer solves: allocated
// on the first such solve if they fit in the free device memory with 1 GiB to spare, else
// never (the solves then pass each problem through its stream's staging arrays).
bool ensure_resident(ftoep_plan pl) {
  if (pl->res_f) return true;
  if (pl->res_tried) return false;
  pl->res_tried = true;
  int64_t need = 0;
  for (const auto& g : pl->groups) {
    int64_t n = 0;
    for (int i : g.probs) n += pl->probs[i].M * pl->probs[i].N;
    need = std::max(need, n);
  }
  const size_t bytes = (size_t)need * sizeof(double);
  size_t free_b = 0, total_b = 0;
  if (need == 0 || cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (2 * bytes + (size_t(1) << 30) > free_b) return false;
  void *a = nullptr, *b = nullptr;
  if (cudaMalloc(&a, bytes) != cudaSuccess || cudaMalloc(&b, bytes) != cudaSuccess) {
    cudaGetLastError();
    if (a) cudaFree(a);
    return false;
  }
  pl->allocs.push_back(a);
  pl->allocs.push_back(b);
  pl->res_f = (double*)a;
  pl->res_u = (double*)b;
  return true;
}

// Make the internal streams wait for the caller's stream.
ftoep_status fork_streams(ftoep_plan pl) {
  if (pl->ws.size() == 1 && !pl->ws[0].own) return FTOEP_OK;
  CK(cudaEventRecord(pl->fork, pl->stream));
  for (auto& w : pl->ws) CK(cudaStreamWaitEvent(w.st, pl->fork, 0));
  return FTOEP_OK;
}

// Make the caller's stream wait for the internal streams.
ftoep_status join_streams(ftoep_plan pl) {
  if (pl->ws.size() == 1 && !pl->ws[0].own) return FTOEP_OK;
  for (auto& w : pl->ws) {
    CK(cudaEventRecord(w.done, w.st));
    CK(cudaStreamWaitEvent(pl->stream, w.done, 0));
  }
  return FTOEP_OK;
}

// Forward transform of (br, bi) (length P, a power of two), in the bit-reversed order of the
// device decimation-in-frequency FFT and divided by P.  Host long double.
std::vector<std::complex<long double>> dif_spectrum(std::vector<long double> br, std::vector<long double> bi) {
  const int64_t P = (int64_t)br.size();
  const long double pi = 3.141592653589793238462643383279502884L;
  // radix-2 decimation in frequency, natural in, bit-reversed out (same permutation as fft_dif)
  for (int64_t len = P; len >= 2; len >>= 1) {
    const int64_t half = len / 2;
    for (int64_t i = 0; i < half; ++i) {
      const long double a = -2.0L * pi * (long double)i / (long double)len;
      const long double wr = cosl(a), wi = sinl(a);
      for (int64_t s0 = 0; s0 < P; s0 += len) {
        const int64_t x = s0 + i, y = s0 + i + half;
        const long double ur = br[x], ui = bi[x], vr = br[y], vi = bi[y];
        br[x] = ur + vr;
        bi[x] = ui + vi;
        const long double dr = ur - vr, di = ui - vi;
        br[y] = dr * wr - di * wi;
        bi[y] = dr * wi + di * wr;
      }
    }
  }
  std::vector<std::complex<long double>> out(P);
  for (int64_t k = 0; k < P; ++k) out[k] = std::complex<long double>(br[k] / P, bi[k] / P);
  return out;
}

// dif_spectrum of b_m = conj(c_|m|) (|m| < L) wrapped to length P.
std::vector<std::complex<long double>> chirp_kernel_spectrum(const std::vector<long double>& cr,
                                                             const std::vector<long double>& ci, int64_t P) {
  const int64_t L = (int64_t)cr.size();
  std::vector<long double> br(P, 0.0L), bi(P, 0.0L);
  for (int64_t m = 0; m < L; ++m) {
    br[m] = cr[m];
    bi[m] = -ci[m];
    if (m > 0) {
      br[P - m] = cr[m];
      bi[P - m] = -ci[m];
    }
  }
  return dif_spectrum(std::move(br), std::move(bi));
}

// Chirp c_n = exp(-i pi n^2 / L), n < L, with n^2 reduced mod 2L exactly.  Host long double.
void chirp_of(int64_t L, std::vector<long double>& cr, std::vector<long double>& ci) {
  const long double pi = 3.141592653589793238462643383279502884L;
  cr.resize(L);
  ci.resize(L);
  for (int64_t n = 0; n < L; ++n) {
    const int64_t r = (n * n) % (2 * L);
    const long double ang = -pi * (long double)r / (long double)L;
    cr[n] = cosl(ang);
    ci[n] = sinl(ang);
  }
}

// Tables of the sine transform of a problem with K = M+1 not a power of two:
//   double (folded half-length form, a DFT of length L = K): chirp, kernel spectrum of length
//     P >= 2K - 1, fold factors sin(pi j/K), j <= K/2;
//   float (the odd extension, a DFT of length L = 2K, at k = 1 .. K-1 as a convolution minus a
//     correlation of length P >= 2K - 3): chirp, the two kernel spectra G1, G2 interleaved.
//     With w_p = x_{p+1} c_{p+1} (p = 0 .. K-2) the sum over the odd extension is
//       sum_p w_p conj(c_{k-1-p}) - sum_p w_p conj(c_{k+1+p}) = (w * g1)_k - (w~ * g2)_k,
//     g1_m = conj(c_{m-1}), m in [-K+3, K-1];  g2_m = conj(c_{m+1}), m in [1, 2K-3];
//     w~_q = w_{-q}, whose transform is W at -k.  Each range holds 2K - 3 values, so P >= 2K - 3
//     keeps the outputs k = 1 .. K-1 free of wrap-around.
ftoep_status build_bluestein(ftoep_plan pl, Prob& pb) {
  const int64_t K = pb.M + 1;
  const long double pi = 3.141592653589793238462643383279502884L;
  std::vector<long double> cr, ci;
  {  // double, folded
    const int64_t L = K;
    pb.logP64 = ilog2(2 * L - 1);
    const int64_t P = int64_t(1) << pb.logP64;
    chirp_of(L, cr, ci);
    const auto bs = chirp_kernel_spectrum(cr, ci, P);
    std::vector<double2> c64(L), b64(P);
    for (int64_t n = 0; n < L; ++n) c64[n] = make_double2((double)cr[n], (double)ci[n]);
    for (int64_t k = 0; k < P; ++k) b64[k] = make_double2((double)bs[k].real(), (double)bs[k].imag());
    const int64_t Q = K / 2;
    std::vector<double> s64(Q + 1);
    for (int64_t j = 0; j <= Q; ++j) s64[j] = (double)sinl(pi * (long double)j / (long double)K);
    ALLOC(pb.chirp64, L * sizeof(double2));
    ALLOC(pb.bspec64, P * sizeof(double2));
    ALLOC(pb.sinv64, (Q + 1) * sizeof(double));
    CK(cudaMemcpy(pb.chirp64, c64.data(), L * sizeof(double2), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(pb.bspec64, b64.data(), P * sizeof(double2), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(pb.sinv64, s64.data(), (Q + 1) * sizeof(double), cudaMemcpyHostToDevice));
  }
  {  // float, odd extension by a convolution and a correlation
    const int64_t L = 2 * K;
    pb.logP32 = std::max(4, ilog2(2 * K - 3));
    const int64_t P = int64_t(1) << pb.logP32;
    chirp_of(L, cr, ci);
    std::vector<long double> g1r(P, 0.0L), g1i(P, 0.0L), g2r(P, 0.0L), g2i(P, 0.0L);
    for (int64_t m = 3 - K; m <= K - 1; ++m) {
      const int64_t c = m >= 1 ? m - 1 : 1 - m, pos = m >= 0 ? m : P + m;
      g1r[pos] = cr[c];
      g1i[pos] = -ci[c];
    }
    for (int64_t m = 1; m <= 2 * K - 3; ++m) {
      g2r[m % P] = cr[m + 1];
      g2i[m % P] = -ci[m + 1];
    }
    const auto s1 = dif_spectrum(std::move(g1r), std::move(g1i));
    const auto s2 = dif_spectrum(std::move(g2r), std::move(g2i));
    std::vector<float2> c32(L);
    std::vector<float4> g32(P);
    for (int64_t n = 0; n < L; ++n) c32[n] = make_float2((float)cr[n], (float)ci[n]);
    for (int64_t k = 0; k < P; ++k)
      g32[k] = make_float4((float)s1[k].real(), (float)s1[k].imag(), (float)s2[k].real(), (float)s2[k].imag());
    ALLOC(pb.chirp32, L * sizeof(float2));
    ALLOC(pb.bspec32, P * sizeof(float4));
    CK(cudaMemcpy(pb.chirp32, c32.data(), L * sizeof(float2), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(pb.bspec32, g32.data(), P * sizeof(float4), cudaMemcpyHostToDevice));
  }
  pb.bluestein = true;
  return FTOEP_OK;
}

// h = first B entries of T_m^-1 e_1 for every mode (double substitution kernel on the
// unit impulse), then the per-pair spectra C1, C2 in precision `pr`.
ftoep_status build_block_inverse(ftoep_plan pl, Ws& w, Prob& pb, Prec pr, void** c1, void** c2) {
  cudaStream_t st = w.st;
  const int64_t n = 2 * (int64_t)pb.B;
  ALLOC(*c1, (size_t)pb.P * n * velem(pr));  // C1 and C2 share one Hermitian-packed array
  *c2 = nullptr;
  double2* z = (double2*)w.z;
  LAUNCH(FTOEP_K_OTHER, launch_unit_impulse(z, pb.Np, pb.P, pb.B, st));
  CK(cudaMemsetAsync(w.prefix, 0, (size_t)pb.P * sizeof(double2), st));
  BlockArgs ba{};
  ba.z = z;
  ba.ld = pb.Np;
  ba.npairs = pb.P;
  ba.t0 = 0;
  ba.B = pb.B;
  ba.L = pb.L;
  ba.Sf = pb.Sf;
  ba.a = pb.e;
  ba.invdiag = pb.invdiag;
  ba.lamtau = pb.lamtau;
  ba.prefix = w.prefix;
  ba.spec = pb.spec64;
  ba.tw = pl->tw64;
  LAUNCH(FTOEP_K_OTHER, launch_block_solve(P64, ba, st));
  InvSpecArgs is{};
  is.h = z;
  is.ldh = pb.Np;
  is.npairs = pb.P;
  is.B = pb.B;
  is.logB = ilog2(pb.B);
  is.c1 = *c1;
  is.c2 = *c2;
  is.tw64 = pl->tw64;
  LAUNCH(FTOEP_K_OTHER, launch_inverse_spectrum(pr, is, st));
  return FTOEP_OK;
}

// Inverse-series solve set-up: h_m = T_m^-1 e_1 over [0, N) for every mode by the double
// half-split solve of a unit impulse, then the packed spectra of the pairs (length 2 Np,
// four-step order, solve precision), in chunks of pairs that fit the stream's scratch.
ftoep_status build_full_inverse(ftoep_plan pl, Ws& w, Prob& pb) {
  cudaStream_t st = w.st;
  TRY(ensure_level_ws(pl, w));
  if (!pb.c1_64) TRY(build_block_inverse(pl, w, pb, P64, (void**)&pb.c1_64, (void**)&pb.c2_64));
  double2* z = (double2*)w.z;
  LAUNCH(FTOEP_K_OTHER, launch_unit_impulse(z, pb.Np, pb.P, (int)pb.ncols, st));
  Prob q = pb;
  q.prec = P64;
  q.finv = false;
  q.c1 = pb.c1_64;
  q.c2 = pb.c2_64;
  TRY(solve_pairs(pl, w, q, P64, z, pb.spec64));
  const int64_t n = 2 * pb.Np;
  ALLOC(pb.cinv, (size_t)pb.P * n * velem(pb.prec));
  const int64_t chunk = std::max<int64_t>(1, (int64_t)(pl->scr_el / (size_t)n));  // double2 scratch
  for (int64_t p0 = 0; p0 < pb.P; p0 += chunk) {
    FinvSpecArgs fs{};
    fs.h = z + p0 * pb.Np;
    fs.ld = pb.Np;
    fs.N = pb.N;
    fs.npairs = std::min<int64_t>(chunk, pb.P - p0);
    fs.logn = pb.logNp + 1;
    fs.scratch64 = (double2*)w.scratch;
    fs.cs = (char*)pb.cinv + (size_t)p0 * n * velem(pb.prec);
    fs.tw64 = pl->tw64;
    LAUNCH(FTOEP_K_OTHER, launch_finv_spectrum(pb.prec, fs, st));
  }
  return FTOEP_OK;
}

ftoep_status setup_problem(ftoep_plan pl, Prob& pb) {
  const int64_t N = pb.N, Np = pb.Np;
  pb.h_a.resize(Np);
  pb.h_dadg.resize(Np);
  scheme_weights(pb.tk, pb.d.gamma, pb.tau, Np, pb.h_a.data(), pb.h_dadg.data());
  std::vector<double> wu0(N), wphi(N), he(Np);
  initial_weights(pb.tk, pb.d.gamma, pb.tau, N, wu0.data(), wphi.data());
  difference_weights(pb.tk, pb.d.gamma, pb.tau, Np, he.data());
  std::vector<double2> invd(pb.P), lt(pb.P);
  for (int64_t p = 0; p < pb.P; ++p) {
    double lam[2];
    for (int q = 0; q < 2; ++q) {
      // pair p: modes p+1 and M-p (sine transform); lines 2p, 2p+1 (no transform)
      const int64_t m = q == 0 ? p + 1 : pb.M - p;
      if (pb.d.space) {
        const double sn = std::sin((double)m * 3.14159265358979323846 / (2.0 * (double)(pb.M + 1)));
        lam[q] = 4.0 / (pb.h * pb.h) * sn * sn;
      } else {
        lam[q] = pb.d.lambda;
      }
    }
    // difference form per mode: E + lambda tau (1 - (1 - sw) I); only the diagonal
    // carries sw (the Crank-Nicolson average puts half of the level-n spatial term on
    // level n-1, whose u^{n-1} = u^n - tau v^n)
    invd[p] = make_double2(1.0 / (he[0] + pb.sw * lam[0] * pb.tau), 1.0 / (he[0] + pb.sw * lam[1] * pb.tau));
    lt[p] = make_double2(lam[0] * pb.tau, lam[1] * pb.tau);
  }
  ALLOC(pb.a, Np * sizeof(double));
  ALLOC(pb.dadg, Np * sizeof(double));
  ALLOC(pb.e, Np * sizeof(double));
  ALLOC(pb.wu0, N * sizeof(double));
  ALLOC(pb.wphi, N * sizeof(double));
  ALLOC(pb.invdiag, pb.P * sizeof(double2));
  ALLOC(pb.lamtau, pb.P * sizeof(double2));
  CK(cudaMemcpy(pb.a, pb.h_a.data(), Np * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(pb.dadg, pb.h_dadg.data(), Np * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(pb.e, he.data(), Np * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(pb.wu0, wu0.data(), N * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(pb.wphi, wphi.data(), N * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(pb.invdiag, invd.data(), pb.P * sizeof(double2), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(pb.lamtau, lt.data(), pb.P * sizeof(double2), cudaMemcpyHostToDevice));
  if (pb.d.space && !is_pow2(pb.M + 1)) TRY(build_bluestein(pl, pb));
  Ws& w = pl->ws[0];
  const size_t nspec = pb.Sf <= Np / 2 ? (size_t)2 * (Np - pb.Sf) : 0;
  if (nspec) {
    ALLOC(pb.spec, nspec * velem(pb.prec));
    TRY(build_solve_spectra(pl, w, pb, pb.prec, pb.spec));
    if (pb.prec == P64) {
      pb.spec64 = (double2*)pb.spec;
    } else {
      ALLOC(pb.spec64, nspec * sizeof(double2));
      TRY(build_solve_spectra(pl, w, pb, P64, pb.spec64));
    }
  }
  TRY(build_block_inverse(pl, w, pb, pb.prec, &pb.c1, &pb.c2));
  if (pb.prec == P64) {
    pb.c1_64 = (double2*)pb.c1;
    pb.c2_64 = (double2*)pb.c2;
  }
  if (pb.prec == P32) TRY(build_product_spectrum(pl, w, pb, pb.e, &pb.spec_res, PFF));
  if (pb.finv) TRY(build_full_inverse(pl, w, pb));
  return FTOEP_OK;
}

// Work of one pair's chain, in n log2 n units: nblk block solves (length 2B) and the
// cross-block convolutions (length 2s, s = B 2^ctz(v), v = 1 .. nblk-1).
double chain_pair_cost(const Prob& pb) {
  auto c = [](double n) { return n * std::log2(n); };
  double t = pb.nblk * c(2.0 * pb.B);
  for (int v = 1; v < pb.nblk; ++v) t += c(2.0 * (double)((int64_t)pb.B << ctz64(v)));
  return t;
}

size_t pair_bytes(const Prob& pb) { return (size_t)pb.P * pb.Np * velem(pb.prec); }

// Chain schedule set-up: per precision the kernel's shared memory, resident grid and
// four-step scratch; problems in groups whose pair arrays fit the memory budget (longest
// chains first), each group with its device descriptors and its item list (pairs, longest
// chains first); one work counter per chain launch.
ftoep_status setup_chain(ftoep_plan pl) {
  int nsm = 0;
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, pl->device));
  for (int pi = 0; pi < 2; ++pi) {
    const Prec pr = pi == 0 ? P64 : P32;
    int maxB = 0;
    int64_t scr = 0;
    bool any = false;
    for (auto& pb : pl->probs) {
      if (pb.prec != pr || pb.finv) continue;
      any = true;
      maxB = std::max(maxB, pb.B);
      for (int v = 1; v < pb.nblk; ++v) {
        const int64_t n = (int64_t)2 * ((int64_t)pb.B << ctz64(v));
        if (n > nsmem_for(pr)) scr = std::max(scr, n);
      }
    }
    if (!any) continue;
    const size_t smem = chain_smem_bytes(pr, maxB);
    const int nb = chain_blocks_per_sm(pr, smem);
    if (nb < 1) return fail(pl, FTOEP_ECUDA, "chain kernel: no block fits an SM with %zu bytes of shared memory", smem);
    pl->chain_smem[pi] = smem;
    pl->chain_grid[pi] = nb * nsm;
    pl->chain_scr_el[pi] = scr;
    if (scr) ALLOC(pl->chain_scr[pi], (size_t)pl->chain_grid[pi] * scr * velem(pr));
  }
  // memory budget of one group's pair arrays: half of what is free, at most 32 GiB, at
  // least the largest problem's
  size_t fr = 0, tot = 0;
  CK(cudaMemGetInfo(&fr, &tot));
  size_t budget = std::min<size_t>(fr / 2, (size_t)32 << 30);
  if (const char* eb = getenv("FTOEP_CHAIN_BUDGET")) {  // bytes; a smaller budget, more groups
    const long long v = atoll(eb);
    if (v > 0) budget = std::min<size_t>(budget, (size_t)v);
  }
  std::vector<int> order(pl->probs.size());
  for (size_t i = 0; i < order.size(); ++i) {
    order[i] = (int)i;
    pl->probs[i].pair_cost = chain_pair_cost(pl->probs[i]);
    budget = std::max(budget, pair_bytes(pl->probs[i]) + 256);
  }
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return pl->probs[x].pair_cost > pl->probs[y].pair_cost; });
  size_t gmax = 0;
  for (int i : order) {
    Prob& pb = pl->probs[i];
    if (pb.finv) continue;  // solved on the internal streams, one convolution per pair
    const size_t b = (pair_bytes(pb) + 255) / 256 * 256;
    if (pl->groups.empty() || pl->groups.back().bytes + b > budget) pl->groups.emplace_back();
    ChainGroup& g = pl->groups.back();
    pb.group = (int)pl->groups.size() - 1;
    pb.zbyte = g.bytes;
    g.bytes += b;
    g.probs.push_back(i);
    gmax = std::max(gmax, g.bytes);
  }
  if (gmax) {
    ALLOC(pl->gz, gmax);
    CK(cudaMemset(pl->gz, 0, gmax));
  }
  pl->ncounters = 2 * (int)pl->groups.size();
  ALLOC(pl->counters, (size_t)pl->ncounters * sizeof(unsigned));
  for (auto& g : pl->groups) {
    std::vector<ChainProb> cp(g.probs.size());
    std::vector<int2> items[2];
    for (size_t k = 0; k < g.probs.size(); ++k) {
      const Prob& pb = pl->probs[g.probs[k]];
      ChainProb& c = cp[k];
      c.z = (char*)pl->gz + pb.zbyte;
      c.ld = pb.Np;
      c.c1 = pb.c1;
      c.lamtau = pb.lamtau;
      c.spec = pb.spec;
      c.Sf = pb.Sf;
      c.nblk = pb.nblk;
      c.logB = ilog2(pb.B);
      const int pi = pb.prec == P64 ? 0 : 1;
      for (int64_t q = 0; q < pb.P; ++q) items[pi].push_back(make_int2((int)k, (int)q));
    }
    ALLOC(g.d_probs, cp.size() * sizeof(ChainProb));
    CK(cudaMemcpy(g.d_probs, cp.data(), cp.size() * sizeof(ChainProb), cudaMemcpyHostToDevice));
    for (int pi = 0; pi < 2; ++pi) {
      g.nitems[pi] = (int)items[pi].size();
      if (!g.nitems[pi]) continue;
      ALLOC(g.d_items[pi], items[pi].size() * sizeof(int2));
      CK(cudaMemcpy(g.d_items[pi], items[pi].data(), items[pi].size() * sizeof(int2), cudaMemcpyHostToDevice));
    }
  }
  return FTOEP_OK;
}

}  // namespace

extern "C" {

ftoep_status ftoep_create(ftoep_plan* out, const ftoep_problem* probs, int nprob, const ftoep_tuning* tune,
                          void* cuda_stream) {
  g_create_error.clear();
  if (!out) return fail(nullptr, FTOEP_EINVAL, "out is NULL");
  *out = nullptr;
  if (!probs || nprob < 1) return fail(nullptr, FTOEP_EINVAL, "need at least one problem");
  for (int i = 0; i < nprob; ++i) TRY(validate(probs[i], i, tune));
  ftoep_plan pl = new ftoep_plan_s();
  pl->stream = (cudaStream_t)cuda_stream;
  {  // host-side fault injection (see ftoep_plan_s::fail_after)
    const char* fa = getenv("FTOEP_FAIL_ALLOC_AFTER");
    pl->fail_after = (fa && *fa) ? atol(fa) : -1;
  }
  {  // host-buffer solves always through the staging arrays (no device copies of the fields)
    const char* hs = getenv("FTOEP_HOST_STAGED");
    if (hs && *hs && atol(hs) != 0) pl->res_tried = true;
  }
  ftoep_status st = FTOEP_OK;
  auto bail = [&](ftoep_status s) {
    g_create_error = pl->err;
    ftoep_destroy(pl);
    return s;
  };
  if (cudaGetDevice(&pl->device) != cudaSuccess) {
    cudaGetLastError();
    pl->err = "no CUDA device";
    return bail(FTOEP_ECUDA);
  }
  int64_t maxtw = 8192;
  int64_t foff = 0, voff = 0;
  for (int i = 0; i < nprob; ++i) {
    Prob pb;
    pb.d = probs[i];
    pb.N = pb.d.N;
    pb.M = pb.d.M;
    pb.prec = pb.d.precision == FTOEP_FP64 ? P64 : P32;
    int64_t np = 16;
    while (np < pb.N) np <<= 1;
    pb.Np = np;
    pb.logNp = ilog2(np);
    pb.P = (pb.M + 1) / 2;
    pb.logK2 = pb.d.space ? ilog2(2 * (pb.M + 1)) : 0;
    pb.tau = pb.d.T / (double)pb.N;
    pb.h = pb.d.space ? pb.d.L / (double)(pb.M + 1) : 1.0;
    pb.tk = pb.d.kind == FTOEP_L1_SUBDIFFUSION ? 0 : 1;
    pb.sw = pb.d.kind == FTOEP_L1_HYPERBOLIC_CN ? 0.5 : 1.0;
    pb.scale = scheme_scale(pb.tk, pb.d.gamma, pb.tau);
    const int Bdef = 4096;
    const int Ldef = 16;
    int B = (tune && tune->fft_tile) ? tune->fft_tile : Bdef;
    if (B > np) B = (int)np;
    int L = (tune && tune->leaf) ? tune->leaf : Ldef;
    if (L > B) L = B;
    int Sf = (tune && tune->gemm_max_level) ? 2 * tune->gemm_max_level : 64;
    if (Sf < L) Sf = L;
    pb.B = B;
    pb.L = L;
    pb.Sf = Sf;
    pb.nblk = (int)((pb.N + B - 1) / B);
    pb.ncols = (int64_t)pb.nblk * B;
    pb.foff = foff;
    pb.voff = voff;
    foff += pb.M * pb.N;
    voff += pb.M;
    maxtw = std::max<int64_t>(maxtw, 2 * np);
    if (pb.d.space) {
      maxtw = std::max<int64_t>(maxtw, 2 * (pb.M + 1));
      if (!is_pow2(pb.M + 1)) maxtw = std::max<int64_t>(maxtw, int64_t(1) << ilog2(4 * (pb.M + 1) - 1));
    }
    pl->z_el = std::max<size_t>(pl->z_el, (size_t)pb.P * np);
    pl->mv_el = std::max<size_t>(pl->mv_el, (size_t)pb.P * np);
    pl->r_el = std::max<size_t>(pl->r_el, (size_t)pb.M * pb.N);
    pl->p_el = std::max<size_t>(pl->p_el, (size_t)pb.P);
    pl->v_el = std::max<size_t>(pl->v_el, (size_t)pb.M);
    pb.cost = (double)pb.M * (double)np * (double)(pb.logNp + 1) * (double)(pb.logNp + 1);
    pl->probs.push_back(std::move(pb));
  }
  pl->total_field = foff;
  pl->total_vec = voff;
  // streams: the caller's stream for one problem, else up to kMaxStreams own streams,
  // problems longest first onto the least-loaded one
  const int want = (tune && tune->streams) ? tune->streams : kDefaultStreams;
  const int nstreams = nprob == 1 ? 1 : std::min(nprob, want);
  // inverse-series solve, on request (FTOEP_SOLVER_INVERSE), for problems with more than
  // one time block and a convolution length above the shared-memory one.  The library's
  // choice is the half split: the inverse-series solve rounds once over the whole time axis,
  // so the early, small levels of a growing solution carry the error of the late, large ones
  // (measured: 4.7e-12 of a sub-diffusion problem's checked set in double, gamma 0.2,
  // N = 127953; 4.6e-3 on the first 1024 levels of the mixed wave workload)
  {
    const int solver = tune ? tune->solver : (int)FTOEP_SOLVER_AUTO;
    for (auto& pb : pl->probs) {
      const int64_t n = 2 * pb.Np;
      const bool want = solver == FTOEP_SOLVER_INVERSE ||
                        (solver == FTOEP_SOLVER_INVERSE_MIXED_SUBDIFFUSION && pb.prec != P64 && pb.tk == 0);
      if (want && pb.nblk >= 2 && n > nsmem_for(pb.prec)) pb.finv = true;
    }
    // the solve's four-step scratch holds one pair's 2 Np values at least
    pl->scr_el = pl->z_el;
    for (auto& pb : pl->probs)
      if (pb.finv) pl->scr_el = std::max(pl->scr_el, (size_t)2 * pb.Np);
  }
  pl->ws.resize(nstreams);
  for (int s = 0; s < nstreams; ++s) {
    Ws& w = pl->ws[s];
    if (nstreams == 1) {
      w.st = pl->stream;
    } else {
      if (cudaStreamCreateWithFlags(&w.st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        pl->err = "stream creation failed";
        return bail(FTOEP_ECUDA);
      }
      w.own = true;
    }
    if (cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      pl->err = "event creation failed";
      return bail(FTOEP_ECUDA);
    }
  }
  if (cudaEventCreateWithFlags(&pl->fork, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    pl->err = "event creation failed";
    return bail(FTOEP_ECUDA);
  }
  {
    std::vector<int> order(nprob);
    for (int i = 0; i < nprob; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return pl->probs[x].cost > pl->probs[y].cost; });
    std::vector<double> load(nstreams, 0.0);
    for (int i : order) {
      const int s = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      pl->probs[i].stream = s;
      load[s] += pl->probs[i].cost;
    }
  }
  // twiddles: W_n^k for all n = 2 .. maxtw at offset n-2, from one long-double table
  {
    pl->ntw = maxtw;
    const size_t tot = (size_t)2 * maxtw - 2;
    std::vector<double2> h64;
    std::vector<float2> h32;
    std::vector<float4> hff;
    host_twiddles(maxtw, &h64, &h32, &hff);
    if ((st = dalloc(pl, (void**)&pl->tw64, tot * sizeof(double2))) != FTOEP_OK) return bail(st);
    if ((st = dalloc(pl, (void**)&pl->tw32, tot * sizeof(float2))) != FTOEP_OK) return bail(st);
    if ((st = dalloc(pl, &pl->twff, tot * sizeof(float4))) != FTOEP_OK) return bail(st);
    if (cudaMemcpy(pl->tw64, h64.data(), tot * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(pl->tw32, h32.data(), tot * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(pl->twff, hff.data(), tot * sizeof(float4), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      pl->err = "twiddle upload failed";
      return bail(FTOEP_ECUDA);
    }
  }
  pl->sched = (tune && tune->scheduler) ? tune->scheduler : (nprob > 1 ? FTOEP_SCHED_CHAIN : FTOEP_SCHED_LEVELS);
  for (auto& w : pl->ws) {
    // the chain schedule solves in group pair arrays: the per-level arrays of the streams
    // are allocated on first use (adjoint), except the first stream's, which the set-up
    // of the block inverses uses
    if (pl->sched == FTOEP_SCHED_LEVELS || &w == &pl->ws[0]) {
      if ((st = dalloc(pl, &w.z, pl->z_el * sizeof(double2))) != FTOEP_OK) return bail(st);
      if (cudaMemsetAsync(w.z, 0, pl->z_el * sizeof(double2), w.st) != cudaSuccess) {
        cudaGetLastError();
        pl->err = "workspace clear failed";
        return bail(FTOEP_ECUDA);
      }
    }
    if (pl->sched == FTOEP_SCHED_LEVELS &&
        (st = dalloc(pl, &w.scratch, pl->scr_el * sizeof(double2))) != FTOEP_OK) return bail(st);
    if ((st = dalloc(pl, (void**)&w.zmv, pl->mv_el * sizeof(double2))) != FTOEP_OK) return bail(st);
    if ((st = dalloc(pl, (void**)&w.scratch_mv, 2 * pl->mv_el * sizeof(double2))) != FTOEP_OK) return bail(st);
    if ((st = dalloc(pl, (void**)&w.r, pl->r_el * sizeof(double))) != FTOEP_OK) return bail(st);
    if ((st = dalloc(pl, (void**)&w.prefix, pl->p_el * sizeof(double2))) != FTOEP_OK) return bail(st);
    if ((st = dalloc(pl, (void**)&w.dpart, kDotBlocks * sizeof(double))) != FTOEP_OK) return bail(st);
  }
  if ((st = dalloc(pl, (void**)&pl->dscal, (size_t)nprob * sizeof(double))) != FTOEP_OK) return bail(st);
  for (auto& pb : pl->probs)
    if ((st = setup_problem(pl, pb)) != FTOEP_OK) return bail(st);
  if (pl->sched == FTOEP_SCHED_CHAIN && (st = setup_chain(pl)) != FTOEP_OK) return bail(st);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    pl->err = "plan set-up failed";
    return bail(FTOEP_ECUDA);
  }
  *out = pl;
  return FTOEP_OK;
}

ftoep_status ftoep_problem_solver(ftoep_plan pl, int iprob, int* solver) {
  if (!pl) return fail(nullptr, FTOEP_EINVAL, "plan is NULL");
  if (iprob < 0 || iprob >= (int)pl->probs.size() || !solver) return fail(pl, FTOEP_EINVAL, "iprob out of range or solver NULL");
  *solver = pl->probs[iprob].finv ? FTOEP_SOLVER_INVERSE : FTOEP_SOLVER_HALFSPLIT;
  return FTOEP_OK;
}

ftoep_status ftoep_weights(ftoep_plan pl, int iprob, double* a, double* dadgamma) {
  if (!pl) return fail(nullptr, FTOEP_EINVAL, "plan is NULL");
  if (iprob < 0 || iprob >= (int)pl->probs.size()) return fail(pl, FTOEP_EINVAL, "iprob out of range");
  if (!a) return fail(pl, FTOEP_EINVAL, "a is NULL");
  Prob& pb = pl->probs[iprob];
  CK(cudaMemcpy(a, pb.h_a.data(), pb.N * sizeof(double), cudaMemcpyDefault));
  if (dadgamma) CK(cudaMemcpy(dadgamma, pb.h_dadg.data(), pb.N * sizeof(double), cudaMemcpyDefault));
  return FTOEP_OK;
}

}  // extern "C"

namespace {

// The workspace a problem runs with: its stream's, on that stream -- or, while the
// instrumentation is on, on the caller's stream, so that the event times of the kernel
// classes do not overlap (the workspaces stay distinct; the stream only orders them).
Ws ws_for(ftoep_plan pl, const Prob& pb) {
  Ws w = pl->ws[pb.stream];
  if (pl->prof_on) w.st = pl->stream;
  return w;
}

// Every problem of the plan on its stream, per-level launches, forked from and joined back
// to the caller's.
// One problem with per-level launches on its internal stream and workspace (host
// buffers through the stream's staging arrays).
ftoep_status solve_on_stream(ftoep_plan pl, Prob& pb, const double* f, double* u, const double* u0,
                             const double* phi, bool host) {
  Ws& wr = pl->ws[pb.stream];
  TRY(ensure_level_ws(pl, wr));
  if (host) TRY(ensure_staging(pl, wr));
  Ws w = ws_for(pl, pb);
  cudaStream_t st = w.st;
  const double* pf = f + pb.foff;
  double* pu = u + pb.foff;
  const double* pu0 = u0 ? u0 + pb.voff : nullptr;
  const double* pphi = phi ? phi + pb.voff : nullptr;
  if (host) {
    const size_t bytes = (size_t)pb.M * pb.N * sizeof(double);
    CK(cudaMemcpyAsync(w.stage_in, pf, bytes, cudaMemcpyDefault, st));
    if (pu0) {
      CK(cudaMemcpyAsync(w.stage_v0, pu0, pb.M * sizeof(double), cudaMemcpyDefault, st));
      pu0 = w.stage_v0;
    }
    if (pphi) {
      CK(cudaMemcpyAsync(w.stage_v1, pphi, pb.M * sizeof(double), cudaMemcpyDefault, st));
      pphi = w.stage_v1;
    }
    TRY(solve_problem(pl, w, pb, w.stage_in, w.stage_out, pu0, pphi));
    CK(cudaMemcpyAsync(pu, w.stage_out, bytes, cudaMemcpyDefault, st));
  } else {
    TRY(solve_problem(pl, w, pb, pf, pu, pu0, pphi));
  }
  return FTOEP_OK;
}

ftoep_status solve_all_levels(ftoep_plan pl, const double* f, double* u, const double* u0, const double* phi,
                              bool host) {
  TRY(fork_streams(pl));
  for (auto& pb : pl->probs) TRY(solve_on_stream(pl, pb, f, u, u0, phi, host));
  TRY(join_streams(pl));
  return FTOEP_OK;
}

// One persistent chain launch over the pairs of one precision of a group, on the caller's
// stream (after zeroing its work counter).
ftoep_status chain_launch(ftoep_plan pl, int gi, int pi, int phase) {
  ChainGroup& g = pl->groups[gi];
  if (!g.nitems[pi]) return FTOEP_OK;
  const Prec pr = pi == 0 ? P64 : P32;
  cudaStream_t st = pl->stream;
  unsigned* counter = pl->counters + 2 * gi + phase;
  CK(cudaMemsetAsync(counter, 0, sizeof(unsigned), st));
  ChainArgs a{};
  a.probs = g.d_probs;
  a.items = g.d_items[pi];
  a.nitems = g.nitems[pi];
  a.counter = counter;
  a.scratch = pl->chain_scr[pi];
  a.scratch_per_block = pl->chain_scr_el[pi];
  a.smem_elems = (int)(pl->chain_smem[pi] / velem(pr));
  a.nsmem = nsmem_for(pr);
  a.tw = tw_of(pl, pr);
  const int grid = std::min(pl->chain_grid[pi], g.nitems[pi]);
  LAUNCH(FTOEP_K_CHAIN, launch_chain(pr, a, grid, pl->chain_smem[pi], st));
  return FTOEP_OK;
}

// Host buffers of one problem through its stream's staging arrays.
struct Staged {
  const double *f = nullptr, *u0 = nullptr, *phi = nullptr;
  double* u = nullptr;
};
// (f NULL: only the initial-data vectors.)
ftoep_status stage_inputs(ftoep_plan pl, Ws& w, const Prob& pb, const double* f, const double* u0,
                          const double* phi, Staged* out) {
  cudaStream_t st = w.st;
  if (f) {
    CK(cudaMemcpyAsync(w.stage_in, f, (size_t)pb.M * pb.N * sizeof(double), cudaMemcpyDefault, st));
    out->f = w.stage_in;
  }
  out->u = w.stage_out;
  if (u0) {
    CK(cudaMemcpyAsync(w.stage_v0, u0, pb.M * sizeof(double), cudaMemcpyDefault, st));
    out->u0 = w.stage_v0;
  }
  if (phi) {
    CK(cudaMemcpyAsync(w.stage_v1, phi, pb.M * sizeof(double), cudaMemcpyDefault, st));
    out->phi = w.stage_v1;
  }
  return FTOEP_OK;
}

// Chain schedule: per group of problems whose pair arrays are resident together --
//   1. every problem: right-hand side + forward sine transform into its pair array
//      (internal streams);
//   2. one persistent chain launch per precision solves every pair of the group;
//   3. every problem: inverse transform + time sums (double: done); mixed: residual and
//      its forward transform;
//   4. mixed: one chain launch solves the correction of every pair;
//   5. mixed: inverse transform, u += tau cumsum.
// Host buffers: when the group's fields fit on the device (ensure_resident), f is copied in
// once in step 1 and u out once after its last step, and the steps run on the device
// copies; otherwise every problem goes through its stream's staging arrays one at a time (f
// copied in for steps 1 and 3, u copied out after step 3 and again, updated, after step 5).
ftoep_status solve_all_chain(ftoep_plan pl, const double* f, double* u, const double* u0, const double* phi,
                             bool host) {
  if (host)
    for (auto& w : pl->ws) TRY(ensure_staging(pl, w));
  const bool res = host && ensure_resident(pl);
  // problems with the inverse-series solve: whole solves on the internal streams
  bool any_finv = false;
  for (auto& pb : pl->probs) any_finv |= pb.finv;
  if (any_finv) {
    TRY(fork_streams(pl));
    for (auto& pb : pl->probs)
      if (pb.finv) TRY(solve_on_stream(pl, pb, f, u, u0, phi, host));
    TRY(join_streams(pl));
  }
  for (size_t gi = 0; gi < pl->groups.size(); ++gi) {
    ChainGroup& g = pl->groups[gi];
    bool mixed = false;
    // offsets of the group's problems in the device copies of the fields
    std::vector<int64_t> roff;
    int64_t ro = 0;
    for (int i : g.probs) {
      roff.push_back(ro);
      ro += pl->probs[i].M * pl->probs[i].N;
    }
    TRY(fork_streams(pl));
    for (size_t k = 0; k < g.probs.size(); ++k) {
      Prob& pb = pl->probs[g.probs[k]];
      Ws w = ws_for(pl, pb);
      void* z = (char*)pl->gz + pb.zbyte;
      const double* pu0 = u0 ? u0 + pb.voff : nullptr;
      const double* pphi = phi ? phi + pb.voff : nullptr;
      mixed |= pb.prec != P64;
      if (res) {
        Staged sg;
        TRY(stage_inputs(pl, w, pb, nullptr, pu0, pphi, &sg));
        double* rf = pl->res_f + roff[k];
        CK(cudaMemcpyAsync(rf, f + pb.foff, (size_t)pb.M * pb.N * sizeof(double), cudaMemcpyDefault, w.st));
        TRY(rhs_forward(pl, w, pb, z, rf, sg.u0, sg.phi));
      } else if (host) {
        Staged sg;
        TRY(stage_inputs(pl, w, pb, f + pb.foff, pu0, pphi, &sg));
        TRY(rhs_forward(pl, w, pb, z, sg.f, sg.u0, sg.phi));
      } else {
        TRY(rhs_forward(pl, w, pb, z, f + pb.foff, pu0, pphi));
      }
    }
    TRY(join_streams(pl));
    for (int pi = 0; pi < 2; ++pi) TRY(chain_launch(pl, (int)gi, pi, 0));
    TRY(fork_streams(pl));
    for (size_t k = 0; k < g.probs.size(); ++k) {
      Prob& pb = pl->probs[g.probs[k]];
      Ws w = ws_for(pl, pb);
      void* z = (char*)pl->gz + pb.zbyte;
      const double* pu0 = u0 ? u0 + pb.voff : nullptr;
      const double* pphi = phi ? phi + pb.voff : nullptr;
      if (res) {
        Staged sg;
        TRY(stage_inputs(pl, w, pb, nullptr, pu0, pphi, &sg));
        double* ru = pl->res_u + roff[k];
        TRY(after_first_solve(pl, w, pb, z, pl->res_f + roff[k], ru, sg.u0, sg.phi));
        if (pb.prec == P64)
          CK(cudaMemcpyAsync(u + pb.foff, ru, (size_t)pb.M * pb.N * sizeof(double), cudaMemcpyDefault, w.st));
      } else if (host) {
        Staged sg;
        TRY(stage_inputs(pl, w, pb, f + pb.foff, pu0, pphi, &sg));
        TRY(after_first_solve(pl, w, pb, z, sg.f, sg.u, sg.u0, sg.phi));
        CK(cudaMemcpyAsync(u + pb.foff, sg.u, (size_t)pb.M * pb.N * sizeof(double), cudaMemcpyDefault, w.st));
      } else {
        TRY(after_first_solve(pl, w, pb, z, f + pb.foff, u + pb.foff, pu0, pphi));
      }
    }
    TRY(join_streams(pl));
    if (!mixed) continue;
    TRY(chain_launch(pl, (int)gi, 1, 1));
    TRY(fork_streams(pl));
    for (size_t k = 0; k < g.probs.size(); ++k) {
      Prob& pb = pl->probs[g.probs[k]];
      if (pb.prec == P64) continue;
      Ws w = ws_for(pl, pb);
      void* z = (char*)pl->gz + pb.zbyte;
      if (res) {
        double* ru = pl->res_u + roff[k];
        TRY(after_correction(pl, w, pb, z, ru));
        CK(cudaMemcpyAsync(u + pb.foff, ru, (size_t)pb.M * pb.N * sizeof(double), cudaMemcpyDefault, w.st));
      } else if (host) {
        const size_t bytes = (size_t)pb.M * pb.N * sizeof(double);
        CK(cudaMemcpyAsync(w.stage_out, u + pb.foff, bytes, cudaMemcpyDefault, w.st));
        TRY(after_correction(pl, w, pb, z, w.stage_out));
        CK(cudaMemcpyAsync(u + pb.foff, w.stage_out, bytes, cudaMemcpyDefault, w.st));
      } else {
        TRY(after_correction(pl, w, pb, z, u + pb.foff));
      }
    }
    TRY(join_streams(pl));
  }
  return FTOEP_OK;
}

ftoep_status solve_all(ftoep_plan pl, const double* f, double* u, const double* u0, const double* phi, bool host) {
  if (pl->sched == FTOEP_SCHED_CHAIN) return solve_all_chain(pl, f, u, u0, phi, host);
  return solve_all_levels(pl, f, u, u0, phi, host);
}

constexpr size_t kMaxGraphs = 4;

// Device-pointer solves are replayed from a CUDA graph: the first call with a pointer set
// runs directly (and finishes every lazy set-up), the second is captured -- the fork to
// the internal streams, all kernels of every problem and the join -- and launched, later
// calls launch the captured graph.  Capture and replay run on a root stream of the plan,
// ordered after the caller's stream by an event and joined back by another, so the
// caller's stream may be the legacy default stream.  Not used with host buffers or while
// the instrumentation is on.
ftoep_status capture_solve(ftoep_plan pl, SolveGraph* g, const double* f, double* u, const double* u0,
                           const double* phi) {
  int64_t before[kNumClasses];
  for (int c = 0; c < kNumClasses; ++c) before[c] = pl->launches[c];
  // the root stream stands in for the caller's stream (and for a single problem's stream
  // when that is the caller's) while the sequence is recorded
  cudaStream_t caller = pl->stream;
  std::vector<cudaStream_t> saved;
  for (auto& w : pl->ws) {
    saved.push_back(w.st);
    if (w.st == caller) w.st = pl->gstream;
  }
  pl->stream = pl->gstream;
  ftoep_status st = FTOEP_OK;
  cudaGraph_t graph = nullptr;
  cudaError_t ec = cudaStreamBeginCapture(pl->gstream, cudaStreamCaptureModeThreadLocal);
  if (ec == cudaSuccess) {
    st = solve_all(pl, f, u, u0, phi, false);
    ec = cudaStreamEndCapture(pl->gstream, &graph);
  }
  pl->stream = caller;
  for (size_t i = 0; i < pl->ws.size(); ++i) pl->ws[i].st = saved[i];
  if (st != FTOEP_OK || ec != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return st != FTOEP_OK ? st : fail(pl, FTOEP_ECUDA, "capture of the solve: %s", cudaGetErrorString(ec));
  }
  cudaGraphExec_t exec = nullptr;
  ec = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ec != cudaSuccess) return fail(pl, FTOEP_ECUDA, "graph instantiate: %s", cudaGetErrorString(ec));
  g->exec = exec;
  for (int c = 0; c < kNumClasses; ++c) {
    g->launches[c] = pl->launches[c] - before[c];
    pl->launches[c] = before[c];  // counted at launch below
  }
  return FTOEP_OK;
}

ftoep_status solve_device(ftoep_plan pl, const double* f, double* u, const double* u0, const double* phi) {
  if (pl->prof_on) return solve_all(pl, f, u, u0, phi, false);
  SolveGraph* g = nullptr;
  for (size_t i = 0; i < pl->graphs.size(); ++i) {
    SolveGraph& c = pl->graphs[i];
    if (c.f == f && c.u == u && c.u0 == u0 && c.phi == phi) {
      std::rotate(pl->graphs.begin() + i, pl->graphs.begin() + i + 1, pl->graphs.end());
      g = &pl->graphs.back();
      break;
    }
  }
  if (!g) {
    if (pl->graphs.size() == kMaxGraphs) {
      if (pl->graphs.front().exec) cudaGraphExecDestroy(pl->graphs.front().exec);
      pl->graphs.erase(pl->graphs.begin());
    }
    SolveGraph n;
    n.f = f;
    n.u = u;
    n.u0 = u0;
    n.phi = phi;
    pl->graphs.push_back(n);
    g = &pl->graphs.back();
  }
  if (!g->exec && g->runs++ == 0) return solve_all(pl, f, u, u0, phi, false);
  if (!pl->gstream) {
    CK(cudaStreamCreateWithFlags(&pl->gstream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&pl->gev_in, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&pl->gev_out, cudaEventDisableTiming));
  }
  if (!g->exec) TRY(capture_solve(pl, g, f, u, u0, phi));
  CK(cudaEventRecord(pl->gev_in, pl->stream));
  CK(cudaStreamWaitEvent(pl->gstream, pl->gev_in, 0));
  CK(cudaGraphLaunch(g->exec, pl->gstream));
  CK(cudaEventRecord(pl->gev_out, pl->gstream));
  CK(cudaStreamWaitEvent(pl->stream, pl->gev_out, 0));
  for (int c = 0; c < kNumClasses; ++c) pl->launches[c] += g->launches[c];
  return FTOEP_OK;
}

}  // namespace

extern "C" {

ftoep_status ftoep_solve(ftoep_plan pl, const double* f, double* u, const double* u0, const double* phi) {
  if (!pl) return fail(nullptr, FTOEP_EINVAL, "plan is NULL");
  if (!f || !u) return fail(pl, FTOEP_EINVAL, "f and u must not be NULL");
  const size_t fb = (size_t)pl->total_field * sizeof(double);
  if ((const char*)f < (const char*)u + fb && (const char*)u < (const char*)f + fb)
    return fail(pl, FTOEP_EINVAL, "f and u overlap");
  const bool host = !is_device_ptr(f) || !is_device_ptr(u) || !is_device_ptr(u0) || !is_device_ptr(phi);
  if (!host) return solve_device(pl, f, u, u0, phi);
  TRY(solve_all(pl, f, u, u0, phi, true));
  TRY(sync_plan(pl));
  return FTOEP_OK;
}

ftoep_status ftoep_matvec(ftoep_plan pl, int iprob, const double* x, double* y, int64_t nlines, int transpose) {
  if (!pl) return fail(nullptr, FTOEP_EINVAL, "plan is NULL");
  if (iprob < 0 || iprob >= (int)pl->probs.size()) return fail(pl, FTOEP_EINVAL, "iprob out of range");
  if (!x || !y || nlines < 1) return fail(pl, FTOEP_EINVAL, "x, y must not be NULL and nlines >= 1");
  Prob& pb = pl->probs[iprob];
  Ws& w = pl->ws[0];
  const size_t bytes = (size_t)nlines * pb.N * sizeof(double);
  if ((const char*)x < (const char*)y + bytes && (const char*)y < (const char*)x + bytes)
    return fail(pl, FTOEP_EINVAL, "x and y overlap");
  TRY(fork_streams(pl));
  cudaStream_t st = w.st;
  TRY(build_product_spectrum(pl, w, pb, pb.a, (void**)&pb.spec_mv, P64));
  const bool host = !is_device_ptr(x) || !is_device_ptr(y);
  // lines per chunk: twice the pairs the product workspace holds
  const int64_t chunk = 2 * (int64_t)(pl->mv_el / pb.Np);
  double *sx = nullptr, *sy = nullptr;
  if (host) {
    ALLOC(sx, (size_t)chunk * pb.N * sizeof(double));
    ALLOC(sy, (size_t)chunk * pb.N * sizeof(double));
  }
  for (int64_t l0 = 0; l0 < nlines; l0 += chunk) {
    const int64_t nl = std::min<int64_t>(chunk, nlines - l0);
    const double* xin = x + l0 * pb.N;
    double* yout = y + l0 * pb.N;
    if (host) {
      CK(cudaMemcpyAsync(sx, xin, nl * pb.N * sizeof(double), cudaMemcpyDefault, st));
      xin = sx;
    }
    TRY(product_lines(pl, w, pb, P64, pb.spec_mv, xin, host ? sy : yout, nl, transpose ? 1 : 0));
    if (host) CK(cudaMemcpyAsync(yout, sy, nl * pb.N * sizeof(double), cudaMemcpyDefault, st));
  }
  TRY(join_streams(pl));
  if (host) {
    TRY(sync_plan(pl));
    release(pl, sx);
    release(pl, sy);
  }
  return FTOEP_OK;
}

ftoep_status ftoep_adjoint(ftoep_plan pl, const double* g, const double* u, double* dldf, double* dldgamma) {
  if (!pl) return fail(nullptr, FTOEP_EINVAL, "plan is NULL");
  if (!g || !dldf) return fail(pl, FTOEP_EINVAL, "g and dldf must not be NULL");
  if (dldgamma && !u) return fail(pl, FTOEP_EINVAL, "u is required for the gamma gradient");
  const size_t fb = (size_t)pl->total_field * sizeof(double);
  if ((const char*)g < (const char*)dldf + fb && (const char*)dldf < (const char*)g + fb)
    return fail(pl, FTOEP_EINVAL, "g and dldf overlap");
  const bool host = !is_device_ptr(g) || !is_device_ptr(dldf) || !is_device_ptr(u);
  // spectra needed by the double adjoint (built once, ordered before the solves on the
  // caller's stream through the fork below)
  {
    Ws& w0 = pl->ws[0];
    TRY(fork_streams(pl));
    for (auto& pb : pl->probs) {
      if (!pb.spec64 && pb.Sf <= pb.Np / 2) {
        ALLOC(pb.spec64, (size_t)2 * (pb.Np - pb.Sf) * sizeof(double2));
        TRY(build_solve_spectra(pl, w0, pb, P64, pb.spec64));
      }
      if (!pb.c1_64) TRY(build_block_inverse(pl, w0, pb, P64, (void**)&pb.c1_64, (void**)&pb.c2_64));
      if (dldgamma) TRY(build_product_spectrum(pl, w0, pb, pb.dadg, (void**)&pb.spec_dg, P64));
    }
    TRY(join_streams(pl));
  }
  TRY(fork_streams(pl));
  int ip = 0;
  for (auto& pb : pl->probs) {
    Ws& w = pl->ws[pb.stream];
    cudaStream_t st = w.st;
    const double* pg = g + pb.foff;
    const double* pu = u ? u + pb.foff : nullptr;
    double* pd = dldf + pb.foff;
    if (host) {
      TRY(ensure_staging(pl, w));
      const size_t bytes = (size_t)pb.M * pb.N * sizeof(double);
      CK(cudaMemcpyAsync(w.stage_in, pg, bytes, cudaMemcpyDefault, st));
      if (pu && dldgamma) {
        CK(cudaMemcpyAsync(w.stage_u, pu, bytes, cudaMemcpyDefault, st));
        pu = w.stage_u;
      }
      TRY(adjoint_problem(pl, w, pb, w.stage_in, pu, w.stage_out, dldgamma ? pl->dscal + ip : nullptr));
      CK(cudaMemcpyAsync(pd, w.stage_out, bytes, cudaMemcpyDefault, st));
    } else {
      TRY(adjoint_problem(pl, w, pb, pg, pu, pd, dldgamma ? pl->dscal + ip : nullptr));
    }
    ++ip;
  }
  TRY(join_streams(pl));
  if (dldgamma) {
    std::vector<double> hs(pl->probs.size());
    cudaStream_t st = pl->stream;
    CK(cudaMemcpyAsync(hs.data(), pl->dscal, hs.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    TRY(sync_plan(pl));
    for (size_t i = 0; i < hs.size(); ++i) dldgamma[i] = -hs[i];
  } else if (host) {
    TRY(sync_plan(pl));
  }
  return FTOEP_OK;
}

ftoep_status ftoep_profile(ftoep_plan pl, int enable) {
  if (!pl) return fail(nullptr, FTOEP_EINVAL, "plan is NULL");
  CK(cudaDeviceSynchronize());
  for (auto& pe : pl->pending) {
    pl->evpool.push_back(pe.second.first);
    pl->evpool.push_back(pe.second.second);
  }
  pl->pending.clear();
  for (int c = 0; c < kNumClasses; ++c) {
    pl->launches[c] = 0;
    pl->prof_ms[c] = 0.0;
    pl->prof_ops[c] = 0;
  }
  pl->prof_on = enable != 0;
  return FTOEP_OK;
}

ftoep_status ftoep_profile_read(ftoep_plan pl, int kclass, double* total_ms, int64_t* ops, int64_t* launches) {
  if (!pl) return fail(nullptr, FTOEP_EINVAL, "plan is NULL");
  if (kclass < 0 || kclass >= kNumClasses) return fail(pl, FTOEP_EINVAL, "kernel class out of range");
  CK(cudaDeviceSynchronize());
  for (auto& pe : pl->pending) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, pe.second.first, pe.second.second) == cudaSuccess) {
      pl->prof_ms[pe.first] += ms;
      pl->prof_ops[pe.first] += 1;
    } else {
      cudaGetLastError();
    }
    pl->evpool.push_back(pe.second.first);
    pl->evpool.push_back(pe.second.second);
  }
  pl->pending.clear();
  if (total_ms) *total_ms = pl->prof_ms[kclass];
  if (ops) *ops = pl->prof_ops[kclass];
  if (launches) *launches = pl->launches[kclass];
  return FTOEP_OK;
}

ftoep_status ftoep_autotune(const ftoep_problem* probs, int nprob, void* cuda_stream, ftoep_tuning* out) {
  g_create_error.clear();
  if (!out || !probs || nprob < 1) return fail(nullptr, FTOEP_EINVAL, "autotune: need problems and out");
  for (int i = 0; i < nprob; ++i) TRY(validate(probs[i], i, nullptr));
  // sample: evenly over the problems sorted by size, up to 2^28 unknowns in total
  const int64_t cap = (int64_t)1 << 28;
  std::vector<int> order(nprob);
  for (int i = 0; i < nprob; ++i) order[i] = i;
  std::sort(order.begin(), order.end(),
            [&](int a, int b) { return probs[a].M * probs[a].N < probs[b].M * probs[b].N; });
  int64_t total = 0;
  for (int i = 0; i < nprob; ++i) total += probs[i].M * probs[i].N;
  std::vector<ftoep_problem> sample;
  if (total <= cap) {
    sample.assign(probs, probs + nprob);
  } else {
    int64_t used = 0;
    for (int k = 1; k <= nprob; k *= 2) {  // strides nprob, nprob/2, ... until the cap
      sample.clear();
      used = 0;
      const int stride = std::max(1, nprob / k);
      for (int i = stride / 2; i < nprob; i += stride) {
        const ftoep_problem& q = probs[order[i]];
        if (used + q.M * q.N > cap) continue;
        sample.push_back(q);
        used += q.M * q.N;
      }
      if ((int)sample.size() >= std::min(nprob, 16)) break;
    }
    if (sample.empty()) {  // every problem alone exceeds the cap: the smallest one
      sample.push_back(probs[order[0]]);
    }
  }
  int64_t units = 0;
  for (auto& q : sample) units += q.M * q.N;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double *f = nullptr, *u = nullptr;
  if (cudaMalloc(&f, (size_t)units * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&u, (size_t)units * sizeof(double)) != cudaSuccess) {
    cudaFree(f);
    cudaGetLastError();
    return fail(nullptr, FTOEP_ENOMEM, "autotune: no memory for %lld sample unknowns", (long long)units);
  }
  cudaMemsetAsync(f, 0, (size_t)units * sizeof(double), st);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::vector<ftoep_tuning> cands;
  const int ns_list[] = {2, 4, 8};
  // the half-split solver only: the inverse-series solves trade accuracy (INVERSE) or device
  // memory (their spectra: 8-16 B per unknown x 2 Np/N, which a sample does not show) for
  // time, a choice the caller makes explicitly
  for (int sv : {(int)FTOEP_SOLVER_HALFSPLIT}) {
    for (int B : {1024, 2048, 4096}) {
      for (int sch : {(int)FTOEP_SCHED_LEVELS, (int)FTOEP_SCHED_CHAIN}) {
        if (sample.size() == 1) {
          ftoep_tuning t{};
          t.fft_tile = B;
          t.scheduler = sch;
          t.solver = sv;
          cands.push_back(t);
          continue;
        }
        for (int ns : ns_list) {
          ftoep_tuning t{};
          t.fft_tile = B;
          t.scheduler = sch;
          t.streams = ns;
          t.solver = sv;
          cands.push_back(t);
        }
      }
    }
  }
  float best_ms = -1.0f;
  ftoep_tuning best{};
  ftoep_status status = FTOEP_OK;
  for (const ftoep_tuning& t : cands) {
    ftoep_plan pl = nullptr;
    status = ftoep_create(&pl, sample.data(), (int)sample.size(), &t, cuda_stream);
    if (status != FTOEP_OK) break;
    // direct run, captured run, then two timed replays
    for (int r = 0; r < 2 && status == FTOEP_OK; ++r) status = ftoep_solve(pl, f, u, nullptr, nullptr);
    if (status == FTOEP_OK) cudaEventRecord(e0, st);
    for (int r = 0; r < 2 && status == FTOEP_OK; ++r) status = ftoep_solve(pl, f, u, nullptr, nullptr);
    if (status == FTOEP_OK) {
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (best_ms < 0.0f || ms < best_ms) {
        best_ms = ms;
        best = t;
      }
    } else {
      g_create_error = pl->err;
    }
    ftoep_destroy(pl);
    if (status != FTOEP_OK) break;
  }
  cudaStreamSynchronize(st);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(f);
  cudaFree(u);
  if (status != FTOEP_OK) return status;
  *out = best;
  return FTOEP_OK;
}

// Restarted GMRES (Sec. 3.2) on the space-time system of problem iprob with zero initial
// data: A u = f, A = I_M (x) T + K (x) I_N (the reordered Eq. 21; T the time operator's first
// column a, K the spatial operator, for the Crank-Nicolson kind averaged over two levels).
// Products: T by circulant embedding (product_lines), K by a stencil kernel.  Arnoldi with
// classical Gram-Schmidt applied twice, Givens rotations on the host.
ftoep_status ftoep_gmres(ftoep_plan pl, int iprob, const double* f, double* u, int restart, double tol, int maxit,
                         int* iters, double* relres) {
  if (!pl) return fail(nullptr, FTOEP_EINVAL, "plan is NULL");
  if (iprob < 0 || iprob >= (int)pl->probs.size()) return fail(pl, FTOEP_EINVAL, "iprob out of range");
  if (!f || !u) return fail(pl, FTOEP_EINVAL, "f and u must not be NULL");
  if (restart < 1 || restart > kMaxBasis) return fail(pl, FTOEP_EINVAL, "restart must be in [1, %d]", kMaxBasis);
  if (!(tol > 0.0) || maxit < 1) return fail(pl, FTOEP_EINVAL, "tol must be > 0 and maxit >= 1");
  Prob& pb = pl->probs[iprob];
  const int64_t M = pb.M, N = pb.N, L = M * N;
  cudaStream_t st = pl->stream;
  Ws w = pl->ws[0];
  w.st = st;
  TRY(build_product_spectrum(pl, w, pb, pb.a, (void**)&pb.spec_mv, P64));
  const bool host = !is_device_ptr(f) || !is_device_ptr(u);
  const int m = restart;
  constexpr int nb = 256;
  double *V = nullptr, *wv = nullptr, *fd = nullptr, *ud = nullptr, *partial = nullptr, *cdev = nullptr;
  ftoep_status status = FTOEP_OK;
  auto cleanup = [&]() {
    release(pl, V);
    release(pl, wv);
    release(pl, fd);
    release(pl, ud);
    release(pl, partial);
    release(pl, cdev);
  };
#define GTRY(expr)                 \
  do {                             \
    if ((status = (expr)) != FTOEP_OK) { \
      cleanup();                   \
      return status;               \
    }                              \
  } while (0)
  GTRY(dalloc(pl, (void**)&V, (size_t)(m + 1) * L * sizeof(double)));
  GTRY(dalloc(pl, (void**)&wv, (size_t)L * sizeof(double)));
  GTRY(dalloc(pl, (void**)&partial, (size_t)(kMaxBasis + 1) * nb * sizeof(double)));
  GTRY(dalloc(pl, (void**)&cdev, (size_t)(kMaxBasis + 1) * sizeof(double)));
  const double* fin = f;
  double* x = u;
  if (host) {
    GTRY(dalloc(pl, (void**)&fd, (size_t)L * sizeof(double)));
    GTRY(dalloc(pl, (void**)&ud, (size_t)L * sizeof(double)));
    if (cudaMemcpyAsync(fd, f, (size_t)L * sizeof(double), cudaMemcpyDefault, st) != cudaSuccess ||
        cudaMemcpyAsync(ud, u, (size_t)L * sizeof(double), cudaMemcpyDefault, st) != cudaSuccess) {
      cudaGetLastError();
      cleanup();
      return fail(pl, FTOEP_ECUDA, "gmres: staging copy failed");
    }
    fin = fd;
    x = ud;
  }
  const double inv_h2 = 1.0 / (pb.h * pb.h);
  auto Amul = [&](const double* xin, double* y) -> ftoep_status {
    TRY(product_lines(pl, w, pb, P64, pb.spec_mv, xin, y, M, 0));
    LAUNCH(FTOEP_K_OTHER, launch_space_add(y, xin, M, N, pb.d.space, inv_h2, pb.d.lambda, pb.sw, st));
    return FTOEP_OK;
  };
  std::vector<double> hp((size_t)(kMaxBasis + 1) * nb);
  auto dots = [&](const double* Vb, int k, const double* xin, double* out) -> ftoep_status {
    LAUNCH(FTOEP_K_OTHER, launch_mdot(Vb, L, k, xin, L, partial, nb, st));
    CK(cudaMemcpyAsync(hp.data(), partial, (size_t)k * nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int i = 0; i < k; ++i) {
      double acc = 0.0;
      for (int b = 0; b < nb; ++b) acc += hp[(size_t)i * nb + b];
      out[i] = acc;
    }
    return FTOEP_OK;
  };
  auto norm = [&](const double* xin, double* out) -> ftoep_status {
    double d = 0.0;
    TRY(dots(xin, 1, xin, &d));
    *out = std::sqrt(std::max(d, 0.0));
    return FTOEP_OK;
  };
  auto Vc = [&](int i) { return V + (int64_t)i * L; };
  double bnorm = 0.0, beta = 0.0;
  GTRY(norm(fin, &bnorm));
  std::vector<double> R((size_t)m * (m + 1), 0.0), cs(m), sn(m), g(m + 1), y(m), h(m + 1), c(m + 1);
  int it = 0;
  while (true) {
    // true residual of the current iterate
    GTRY(Amul(x, wv));
    LAUNCH(FTOEP_K_OTHER, launch_lincomb(Vc(0), 1.0, fin, -1.0, wv, L, st));
    GTRY(norm(Vc(0), &beta));
    if (bnorm == 0.0 || beta <= tol * bnorm || it >= maxit) break;
    LAUNCH(FTOEP_K_OTHER, launch_lincomb(Vc(0), 1.0 / beta, Vc(0), 0.0, nullptr, L, st));
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int j = 0;
    while (j < m && it < maxit) {
      GTRY(Amul(Vc(j), wv));
      std::fill(h.begin(), h.end(), 0.0);
      for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt, twice
        GTRY(dots(V, j + 1, wv, c.data()));
        for (int i = 0; i <= j; ++i) {
          h[i] += c[i];
          c[i] = -c[i];
        }
        CK(cudaMemcpyAsync(cdev, c.data(), (size_t)(j + 1) * sizeof(double), cudaMemcpyHostToDevice, st));
        LAUNCH(FTOEP_K_OTHER, launch_maxpy(wv, V, L, j + 1, cdev, L, st));
      }
      double hn = 0.0;
      GTRY(norm(wv, &hn));
      h[j + 1] = hn;
      if (hn > 0.0) LAUNCH(FTOEP_K_OTHER, launch_lincomb(Vc(j + 1), 1.0 / hn, wv, 0.0, nullptr, L, st));
      for (int i = 0; i < j; ++i) {  // earlier rotations on the new column
        const double a = cs[i] * h[i] + sn[i] * h[i + 1];
        h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
        h[i] = a;
      }
      const double rr = std::hypot(h[j], h[j + 1]);
      cs[j] = rr > 0.0 ? h[j] / rr : 1.0;
      sn[j] = rr > 0.0 ? h[j + 1] / rr : 0.0;
      h[j] = rr;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      for (int i = 0; i <= j; ++i) R[(size_t)i * m + j] = h[i];
      ++j;
      ++it;
      if (std::fabs(g[j]) <= tol * bnorm || hn == 0.0) break;
    }
    for (int i = j - 1; i >= 0; --i) {  // R y = g, upper triangular
      double acc = g[i];
      for (int k = i + 1; k < j; ++k) acc -= R[(size_t)i * m + k] * y[k];
      y[i] = R[(size_t)i * m + i] != 0.0 ? acc / R[(size_t)i * m + i] : 0.0;
    }
    CK(cudaMemcpyAsync(cdev, y.data(), (size_t)j * sizeof(double), cudaMemcpyHostToDevice, st));
    LAUNCH(FTOEP_K_OTHER, launch_maxpy(x, V, L, j, cdev, L, st));
  }
  if (host && cudaMemcpyAsync(u, ud, (size_t)L * sizeof(double), cudaMemcpyDefault, st) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return fail(pl, FTOEP_ECUDA, "gmres: copy out failed");
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return fail(pl, FTOEP_ECUDA, "gmres: stream synchronize failed");
  }
#undef GTRY
  cleanup();
  if (iters) *iters = it;
  if (relres) *relres = bnorm > 0.0 ? beta / bnorm : 0.0;
  return FTOEP_OK;
}

// Advection sweeps of Sec. 3 (the fast procedure: space order, Figure 2).  Node i = 1..M solves
// the lower-triangular Toeplitz system of one line, A-tilde U_i = B U_{i-1} + F_i:
//   scheme 2: (c L1 + I/h) U_i = (I/h - c L1) U_{i-1} + F_i, c = mu/2; times 2, the scalar
//             sub-diffusion operator A = mu L1 + (2/h) I and B = (2/h) I - mu L1;
//   scheme 3: (c W + I/h) U_i = U_{i-1}/h + F_i: A = c W + (1/h) I, B = (1/h) I.
// Lower-triangular Toeplitz matrices commute, so U_i = G U_{i-1} + V_i with G = A^-1 B (lower-
// triangular Toeplitz, first column g = A^-1 b, b = B e_1) and V_i = A^-1 F_i.  The recursion
// over i is a linear scan: after the rounds d = 1, 2, 4, ... < M of U_i += G^d U_{i-d} (every
// i >= d at once, from the previous round's values) U_i = sum_{k<=i} G^{i-k} V_k.  So the sweep
// is one batched solve of all M lines (the library's scalar solve, lambda = 2/h resp. 1/h),
// the solve of b, and ceil(log2 M) rounds of a batched circulant-embedded product (Sec. 3.1)
// with the first column of G^d (squared from round to round), instead of M dependent solves.
// Initial data enter the right-hand sides through the plan's initial-data weights (the u-form
// rows; the solves themselves with zero initial value).
ftoep_status ftoep_advection_sweep(int scheme, double gamma, double T, double L, int64_t N, int64_t M,
                                   const double* f, const double* u0, const double* phi, double* u, int precision,
                                   void* cuda_stream) {
  g_create_error.clear();
  if (scheme != 2 && scheme != 3) return fail(nullptr, FTOEP_EINVAL, "advection sweep: scheme %d unknown", scheme);
  if (scheme == 2 && !(gamma > 0.0 && gamma < 1.0))
    return fail(nullptr, FTOEP_EINVAL, "advection sweep: scheme 2 needs gamma in (0,1), got %g", gamma);
  if (scheme == 3 && !(gamma > 1.0 && gamma < 2.0))
    return fail(nullptr, FTOEP_EINVAL, "advection sweep: scheme 3 needs gamma in (1,2), got %g", gamma);
  if (N < 1 || M < 1 || !f || !u || !(T > 0.0) || !(L > 0.0) ||
      (precision != FTOEP_FP64 && precision != FTOEP_MIXED))
    return fail(nullptr, FTOEP_EINVAL, "advection sweep: N, M >= 1, f, u not NULL, T, L > 0, precision FP64/MIXED");
  const double h = L / (double)M;
  ftoep_problem d{};
  d.kind = scheme == 2 ? FTOEP_L1_SUBDIFFUSION : FTOEP_L1_HYPERBOLIC;
  d.space = FTOEP_SPACE_NONE;
  d.precision = precision;
  d.gamma = gamma;
  d.T = T;
  d.L = 1.0;
  d.lambda = scheme == 2 ? 2.0 / h : 1.0 / h;
  d.N = N;
  d.M = M;  // M independent lines of the scalar problem
  ftoep_plan pl = nullptr;
  TRY(ftoep_create(&pl, &d, 1, nullptr, cuda_stream));
  ftoep_status status = FTOEP_OK;
  {
    Prob& pb = pl->probs[0];
    Ws& w = pl->ws[0];
    cudaStream_t st = w.st;
    const int64_t LN = M * N;
    const bool host = !is_device_ptr(f) || !is_device_ptr(u) || !is_device_ptr(u0) || !is_device_ptr(phi);
    auto run = [&]() -> ftoep_status {
      std::vector<double> hu0(u0 ? M : 0), hphi(phi ? M : 0), s0(M, 0.0), s1(M, 0.0);
      if (u0) CK(cudaMemcpy(hu0.data(), u0, M * sizeof(double), cudaMemcpyDefault));
      if (phi) CK(cudaMemcpy(hphi.data(), phi, M * sizeof(double), cudaMemcpyDefault));
      for (int64_t i = 0; i < M; ++i) {
        if (u0) s0[i] = scheme == 2 ? hu0[i] + (i > 0 ? hu0[i - 1] : 0.0) : hu0[i];
        if (phi && scheme == 3) s1[i] = hphi[i];
      }
      TRY(ensure_level_ws(pl, w));
      double *fd = nullptr, *rhs = nullptr, *V = nullptr, *U0 = nullptr, *U1 = nullptr, *Tm = nullptr;
      double *gcol = nullptr, *s0d = nullptr, *s1d = nullptr;
      double2* spec = nullptr;
      ALLOC(rhs, LN * sizeof(double));
      ALLOC(V, LN * sizeof(double));
      ALLOC(U0, LN * sizeof(double));
      ALLOC(U1, LN * sizeof(double));
      ALLOC(Tm, LN * sizeof(double));
      ALLOC(gcol, 2 * N * sizeof(double));
      ALLOC(s0d, M * sizeof(double));
      ALLOC(s1d, M * sizeof(double));
      ALLOC(spec, 2 * pb.Np * sizeof(double2));
      CK(cudaMemcpyAsync(s0d, s0.data(), M * sizeof(double), cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(s1d, s1.data(), M * sizeof(double), cudaMemcpyHostToDevice, st));
      const double* F = f;
      if (host) {
        ALLOC(fd, LN * sizeof(double));
        CK(cudaMemcpyAsync(fd, f, LN * sizeof(double), cudaMemcpyDefault, st));
        F = fd;
      }
      // V = A^-1 (c F + initial-data terms), all nodes at once
      LAUNCH(FTOEP_K_OTHER, launch_sweep_rhs_lines(rhs, F, u0 ? pb.wu0 : nullptr, s0d,
                                                    (phi && scheme == 3) ? pb.wphi : nullptr, s1d, M, N,
                                                    scheme == 2 ? 2.0 : 1.0, st));
      TRY(solve_problem(pl, w, pb, rhs, V, nullptr, nullptr));
      if (M > 1) {
        // first column of G: A^-1 b on line 0 (the other lines zero)
        std::vector<double> b(N, 0.0);
        b[0] = scheme == 2 ? 2.0 / h : 1.0 / h;
        if (scheme == 2)
          for (int64_t n = 0; n < N; ++n) b[n] -= pb.h_a[n];
        CK(cudaMemsetAsync(rhs, 0, LN * sizeof(double), st));
        CK(cudaMemcpyAsync(rhs, b.data(), N * sizeof(double), cudaMemcpyHostToDevice, st));
        TRY(solve_problem(pl, w, pb, rhs, Tm, nullptr, nullptr));
        CK(cudaMemcpyAsync(gcol, Tm, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
        CK(cudaStreamSynchronize(st));  // b is host memory of this scope
      }
      // scan over the nodes: U_i += G^d U_{i-d}, d = 1, 2, 4, ...
      double* cur = V;
      double* nxt = U0;
      double* spare = U1;
      double* gd = gcol;
      double* gn = gcol + N;
      for (int64_t dd = 1; dd < M; dd *= 2) {
        SpecArgs sa{};
        sa.a = gd;
        sa.lo = 0;
        sa.hi = N;
        sa.logn = pb.logNp + 1;
        sa.nsmem = nsmem_for(P64);
        sa.out = spec;
        sa.tw64 = pl->tw64;
        sa.scratch64 = w.scratch_mv;
        LAUNCH(FTOEP_K_OTHER, launch_spectrum(P64, sa, st));
        TRY(product_lines(pl, w, pb, P64, spec, cur, Tm, M - dd, 0));
        LAUNCH(FTOEP_K_OTHER, launch_shift_add_lines(nxt, cur, Tm, M, N, dd, st));
        if (2 * dd < M) {  // G^(2d) = G^d G^d
          TRY(product_lines(pl, w, pb, P64, spec, gd, gn, 1, 0));
          std::swap(gd, gn);
        }
        double* old = cur;
        cur = nxt;
        nxt = old == V ? spare : old;
      }
      CK(cudaMemcpyAsync(u, cur, LN * sizeof(double), cudaMemcpyDefault, st));
      CK(cudaStreamSynchronize(st));
      return FTOEP_OK;
    };
    status = run();
    if (status != FTOEP_OK) g_create_error = pl->err;
  }
  ftoep_destroy(pl);
  return status;
}

ftoep_status ftoep_sync(ftoep_plan pl) {
  if (!pl) return fail(nullptr, FTOEP_EINVAL, "plan is NULL");
  return sync_plan(pl);
}

ftoep_status ftoep_last_error(ftoep_plan pl, char* buf, size_t n) {
  if (!buf || n == 0) return FTOEP_EINVAL;
  const std::string& s = pl ? pl->err : g_create_error;
  size_t k = std::min(n - 1, s.size());
  memcpy(buf, s.data(), k);
  buf[k] = '\0';
  return FTOEP_OK;
}

ftoep_status ftoep_destroy(ftoep_plan pl) {
  if (!pl) return FTOEP_EINVAL;
  cudaStreamSynchronize(pl->stream);
  for (auto& w : pl->ws) {
    if (w.st) cudaStreamSynchronize(w.st);
  }
  cudaGetLastError();
  for (void* ptr : pl->allocs) cudaFree(ptr);
  for (auto& pe : pl->pending) {
    cudaEventDestroy(pe.second.first);
    cudaEventDestroy(pe.second.second);
  }
  for (cudaEvent_t e : pl->evpool) cudaEventDestroy(e);
  for (auto& w : pl->ws) {
    if (w.done) cudaEventDestroy(w.done);
    if (w.own && w.st) cudaStreamDestroy(w.st);
  }
  if (pl->fork) cudaEventDestroy(pl->fork);
  if (pl->gstream) cudaStreamSynchronize(pl->gstream);
  for (auto& g : pl->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (pl->gstream) cudaStreamDestroy(pl->gstream);
  if (pl->gev_in) cudaEventDestroy(pl->gev_in);
  if (pl->gev_out) cudaEventDestroy(pl->gev_out);
  delete pl;
  return FTOEP_OK;
}

}  // extern "C"
