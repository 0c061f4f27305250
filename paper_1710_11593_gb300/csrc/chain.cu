// Persistent per-pair solve: one launch solves every mode pair of every problem of a
// group (the half-split triangular Toeplitz solve of Sec. 3's reordered per-line systems,
// after the sine decoupling).
//
// After the sine transform the mode pairs are independent: nothing couples two pairs
// until the inverse transform.  So one block can run a pair's whole time recursion by
// itself -- for b = 0 .. nblk-1: the block solve of time block b (block_inverse_body),
// then the one cross-block update that becomes due, level s = B * 2^ctz(b+1): a circulant
// convolution of length 2s, in shared memory when it fits, else as a four-step transform
// that the block runs alone through its own slice of a global scratch array.  No block
// ever waits for another, and the running sums of the all-ones part stay in shared memory.
//
// Scheduling: the grid is sized to the blocks that are resident at once; each block takes
// the next (problem, pair) item from a global counter until the list is exhausted.  Items
// are ordered longest chain first (longest-processing-time list scheduling), so the
// launch ends on short chains.  The counter is zeroed on the stream before every launch.
#include "block_inverse_body.cuh"
#include "internal.h"

namespace ftoep {

namespace {

constexpr int kChainThreads = 256;

// Blocks per SM the register budget is sized for: three float blocks (64 KB of shared
// memory each), two double blocks (the double block solve alone takes 128 KB, so one is
// resident; the bound keeps the register count at the per-level kernels' level).
// kInf: elements a thread keeps in flight in the global-memory passes of the bodies.  The
// per-level kernels use 8; here the bodies are calls with the recursion's state around them,
// and 8 (or 4) made every body spill inside its passes (measured: local-memory traffic above
// the kernel's DRAM traffic); with 2 the bodies stay in registers.
#ifndef FTOEP_CHAIN_OCC
#define FTOEP_CHAIN_OCC 3
#endif
#ifndef FTOEP_CHAIN_INF
#define FTOEP_CHAIN_INF 2
#endif
#ifndef FTOEP_CHAIN_CALL
#define FTOEP_CHAIN_CALL __noinline__
#endif
template <typename T> struct ChainOcc { static constexpr int value = FTOEP_CHAIN_OCC; };
template <> struct ChainOcc<double> { static constexpr int value = 2; };
constexpr int kInf = FTOEP_CHAIN_INF;
// kAsync: the first pass of every body takes its input by cp.async into shared memory (one
// block per pair has no other blocks' loads to hide its own latency behind).
#ifndef FTOEP_CHAIN_ASYNC
#define FTOEP_CHAIN_ASYNC 1
#endif
constexpr bool kAsync = FTOEP_CHAIN_ASYNC != 0;

// Each body runs as a call of its own: registers are then allocated per body (as in the
// per-level kernels) instead of across the whole recursion, and the state of the
// recursion lives in shared memory between the calls.
template <typename T>
__device__ FTOEP_CHAIN_CALL void chain_block(Vt<T>* sm, Vt<T>* zg, const Vt<T>* cs, int logB, double2 lt, double2 S, T* red,
                                         double2* S_out, const Vt<T>* tw) {
  block_inverse_body<T, kInf, kAsync>(sm, zg, cs, logB, lt, S, red, S_out, tw);
}
template <typename T>
__device__ FTOEP_CHAIN_CALL void chain_conv_smem(Vt<T>* sm, const Vt<T>* zin, Vt<T>* zo, int logn, const Vt<T>* spec,
                                             const Vt<T>* tw) {
  conv_smem_body<T, kInf, kAsync>(sm, zin, zo, logn, 0, spec, tw);
}
// The whole four-step convolution of one pair (three steps over column and row groups of
// at most cap elements), through the block's scratch slice.
template <typename T>
__device__ FTOEP_CHAIN_CALL void chain_fourstep(Vt<T>* sm, const Vt<T>* zin, Vt<T>* zo, Vt<T>* scr, const Vt<T>* spec,
                                            int logn, int cap, const Vt<T>* tw) {
  typedef Vt<T> V;
  const Split sp = split_of(logn);
  const int C = fourstep_cols_for(sp.logn1, sp.logn2, (int)sizeof(V), cap);
  const int rows = min(cap >> sp.logn2, 1 << sp.logn1);
  for (int c0 = 0; c0 < (1 << sp.logn2); c0 += C) {
    conv_col_fwd_body<T, kInf, kAsync>(sm, zin, scr, sp.logn1, sp.logn2, C, c0, tw);
    __syncthreads();
  }
  for (int r0 = 0; r0 < (1 << sp.logn1); r0 += rows) {
    conv_row_body<T, kInf, kAsync>(sm, scr, spec, sp.logn1, sp.logn2, rows, r0, tw);
    __syncthreads();
  }
  for (int c0 = 0; c0 < (1 << sp.logn2); c0 += C) {
    conv_col_inv_body<T, kInf, kAsync>(sm, scr, zo, sp.logn1, sp.logn2, C, c0, 0, tw);
    __syncthreads();
  }
}

// State of the pair being solved, shared by the block.
struct ChainJob {
  ChainProb P;
  double2 lt;      // lambda tau of the pair's two modes
  double2 S;       // running sums of the solved entries
  int64_t p;       // pair index
  int item;
};

template <typename T>
__global__ void __launch_bounds__(kChainThreads, ChainOcc<T>::value) chain_solve_kernel(ChainArgs A) {
  typedef Vt<T> V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  __shared__ T red[4 * kChainThreads];
  __shared__ ChainJob J;
  for (;;) {
    if (threadIdx.x == 0) {
      const int it = (int)atomicAdd(A.counter, 1u);
      J.item = it;
      if (it < A.nitems) {
        const int2 w = A.items[it];
        J.P = A.probs[w.x];
        J.p = w.y;
        J.lt = J.P.lamtau[w.y];
        J.S = make_double2(0.0, 0.0);
      }
    }
    __syncthreads();
    if (J.item >= A.nitems) return;
    const int nblk = J.P.nblk;
    for (int b = 0; b < nblk; ++b) {
      {
        const int logB = J.P.logB;
        V* row = (V*)J.P.z + J.p * J.P.ld;
        const V* cs = (const V*)J.P.c1 + J.p * ((int64_t)2 << logB);
        const double2 S = J.S;
        const double2 lt = J.lt;
        __syncthreads();  // S read by every thread before thread 0 replaces it
        chain_block<T>(sm, row + ((int64_t)b << logB), cs, logB, lt, S, red, &J.S, (const V*)A.tw);
      }
      __syncthreads();
      const int v = b + 1;
      if (v >= nblk) break;
      const int logB = J.P.logB;
      const int64_t s = (int64_t)1 << (logB + __ffs(v) - 1);  // B * 2^ctz(v)
      const int64_t mid = (int64_t)v << logB;
      const int logn = logB + __ffs(v);                       // log2(2s)
      V* row = (V*)J.P.z + J.p * J.P.ld;
      const V* spec = (const V*)J.P.spec + 2 * (s - J.P.Sf);
      if (2 * s <= A.nsmem) {
        chain_conv_smem<T>(sm, row + (mid - s), row + mid, logn, spec, (const V*)A.tw);
        __syncthreads();
      } else {
        chain_fourstep<T>(sm, row + (mid - s), row + mid, (V*)A.scratch + (int64_t)blockIdx.x * A.scratch_per_block,
                          spec, logn, A.smem_elems, (const V*)A.tw);
      }
    }
    __syncthreads();  // J is rewritten for the next item
  }
}

template <typename T>
const void* chain_fn() {
  return (const void*)chain_solve_kernel<T>;
}

}  // namespace

size_t chain_smem_bytes(Prec prec, int maxB) {
  const size_t el = prec == P64 ? sizeof(double2) : sizeof(float2);
  size_t n = (size_t)2 * maxB;                 // block solve: 2B
  const size_t conv = (size_t)nsmem_for(prec);  // shared-memory convolutions
  if (conv > n) n = conv;
  return n * el;
}

int chain_blocks_per_sm(Prec prec, size_t smem) {
  const void* fn = prec == P64 ? chain_fn<double>() : chain_fn<float>();
  set_smem_once(fn, smem);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kChainThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

int launch_chain(Prec prec, const ChainArgs& a, int grid, size_t smem, cudaStream_t st) {
  if (prec == P64) {
    set_smem_once(chain_fn<double>(), smem);
    chain_solve_kernel<double><<<grid, kChainThreads, smem, st>>>(a);
  } else {
    set_smem_once(chain_fn<float>(), smem);
    chain_solve_kernel<float><<<grid, kChainThreads, smem, st>>>(a);
  }
  return 1;
}

}  // namespace ftoep
