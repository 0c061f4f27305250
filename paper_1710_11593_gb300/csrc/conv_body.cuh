// Device bodies of the circulant convolutions behind every Toeplitz product (Sec. 3.1,
// Eq. be1: C = F^-1 diag(F c) F), shared by the per-level kernels (transforms.cu: one
// launch per level, blocks over pairs and column groups) and the persistent per-pair
// solve (chain.cu: one block runs every level of one pair).
//
// Convolution of one pair row: t = x (*) c over length n = 2^logn, x = the first n/2
// entries of the input row zero-padded; mode 0 (half-split update): out[i] -= t[n/2 + i];
// mode 1 (product): out[i] = t[i]; both for i < n/2.
//
// Shared-memory form (n fits one block's shared memory): the first forward pass reads the
// input half straight from global memory, the last forward pass, the product with the
// kernel spectrum and the first inverse pass run fused in registers, and the last inverse
// pass writes (mode 0: subtracts) the wanted half straight to global.
//
// Four-step form: n = n1*n2, index j = j1*n2 + j2.  Step A transforms C columns (over j1)
// at a time, applies W_n^{j2 k1} and writes the scratch; step B transforms `rows` rows
// (over j2) at a time, multiplies by the spectrum (stored in the same order), inverts the
// rows and removes the twiddle; step C inverts the columns.  Column transforms leave k1 in
// bit-reversed row order, which the twiddles account for.  Column groups map consecutive
// threads to consecutive columns (coalesced global access); the first and last passes of
// every step read or write global memory directly.
#pragma once

#include "fft.cuh"
#include "fftr.cuh"

namespace ftoep {
namespace {

template <typename T>
using Vt = typename VecOf<T>::type;

// Asynchronous global -> shared copy of one element (cp.async, 8 or 16 bytes): the data
// does not pass through registers, so a block can have a whole group's loads in flight.
template <typename V>
__device__ __forceinline__ void async_copy(V* sdst, const V* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  if constexpr (sizeof(V) == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gsrc) : "memory");
  }
}
// Wait for this thread's copies, then for the block's.
__device__ __forceinline__ void async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
}

// Pointwise product of spectrum values with a kernel spectrum in the same storage order
// (the op of fftr_middle): x[j] *= spec[pos0 + j].
template <typename V>
struct SpecMul {
  const V* __restrict__ spec;
  template <class X, class RR>
  __device__ __forceinline__ void operator()(int t, int pos0, X& x, RR) const {
    (void)t;
    static_for<0, RR::value>([&](auto JJ) {
      constexpr int j = decltype(JJ)::value;
      x[j] = cmul(x[j], spec[pos0 + j]);
    });
  }
};

// Read-modify-write storers of the last inverse pass (mode 0: subtract the upper half of
// the cyclic result from the output).
template <typename V>
struct SubUpper {  // zo[e - s] -= v for e >= s
  V* __restrict__ zo;
  int s;
  __device__ __forceinline__ V fetch(int, int e) const { return e >= s ? zo[e - s] : vzero<V>(); }
  __device__ __forceinline__ void operator()(int, int e, const V& v, const V& f) const {
    if (e >= s) zo[e - s] = csub(f, v);
  }
};
template <typename V>
struct SubUpperCols {  // column t: zo[(e - h1) n2 + t] -= v for e >= h1
  V* __restrict__ zo;
  int h1, n2;
  __device__ __forceinline__ V fetch(int t, int e) const {
    return e >= h1 ? zo[(int64_t)(e - h1) * n2 + t] : vzero<V>();
  }
  __device__ __forceinline__ void operator()(int t, int e, const V& v, const V& f) const {
    if (e >= h1) zo[(int64_t)(e - h1) * n2 + t] = csub(f, v);
  }
};

// Whole convolution of one pair row in shared memory sm (n elements).  zin: the input
// half (n/2 entries), zo: the output half.  No barrier at the end.
// ASYNC: the input arrives by cp.async into shared memory and the first pass runs there
// (instead of the first pass reading global memory into registers).
template <typename T, int INF = 8, bool ASYNC = false>
__device__ __forceinline__ void conv_smem_body(Vt<T>* sm, const Vt<T>* __restrict__ zin, Vt<T>* __restrict__ zo,
                                               int logn, int mode, const Vt<T>* __restrict__ spec,
                                               const Vt<T>* __restrict__ tw) {
  typedef Vt<T> V;
  const int s = 1 << (logn - 1);
  const SmLayout L = sm_layout<V>(logn);
  const int np = fftr_npasses<V>(logn);
  if constexpr (ASYNC) {
    for (int e = threadIdx.x; e < s; e += blockDim.x) async_copy(&sm[sm_pos<V>(L, 0, e)], zin + e);
    async_wait_all();
    fftr_pass<V, true>(0, logn, 1, tw, true, SmAt<V>{sm, L}, SmPut<V>{sm, L});
  } else {
    fftr_pass<V, true, false, true, false, INF>(0, logn, 1, tw, true, [&](int, int e) { return zin[e]; },
                                                SmPut<V>{sm, L});
  }
  __syncthreads();
  if (np < 2) {  // a single pass: plain product in shared memory
    for (int k = threadIdx.x; k < 2 * s; k += blockDim.x) {
      const int q = sm_pos<V>(L, 0, k);
      sm[q] = cmul(sm[q], spec[k]);
    }
    __syncthreads();
  } else {
    fftr_passes<V, true>(sm, logn, 1, tw, 1, np - 1, false);
    fftr_middle<V>(sm, logn, 1, SpecMul<V>{spec});
    __syncthreads();
    fftr_passes<V, false>(sm, logn, 1, tw, 1, np - 1, false);
  }
  if (mode == 0) {
    fftr_pass<V, false, false, false, true, INF>(np - 1, logn, 1, tw, false, SmAt<V>{sm, L}, SubUpper<V>{zo, s});
  } else {
    fftr_pass<V, false>(np - 1, logn, 1, tw, false, SmAt<V>{sm, L}, [&](int, int e, const V& v) {
      if (e < s) zo[e] = v;
    });
  }
}

// Four-step step A on columns c0 .. c0+C-1: zin is the pair's input half (row layout
// j1*n2 + j2), sc the pair's scratch (n elements).  nvalid > 0: input entries at index
// >= nvalid are read as zero (the padding of a row whose tail holds other data).  No
// barrier at the end.
template <typename T, int INF = 8, bool ASYNC = false>
__device__ __forceinline__ void conv_col_fwd_body(Vt<T>* sm, const Vt<T>* __restrict__ zin_row,
                                                  Vt<T>* __restrict__ sc_row, int logn1, int logn2, int C, int c0,
                                                  const Vt<T>* __restrict__ tw, int64_t nvalid = 0) {
  typedef Vt<T> V;
  const int n2 = 1 << logn2, logn = logn1 + logn2, n = 1 << logn;
  const V* __restrict__ zin = zin_row + c0;
  V* __restrict__ sc = sc_row + c0;
  const V* __restrict__ twn = tw + (n - 2);
  const SmLayout L = sm_layout<V>(logn1);
  const int np = fftr_npasses<V>(logn1);
  const int64_t nv = nvalid > 0 ? nvalid - c0 : ((int64_t)1 << 62);  // relative to zin
  if constexpr (ASYNC) {  // input half: rows e < n1/2 of the C columns
    const int lc = 31 - __clz(C);
    for (int i = threadIdx.x; i < (C << (logn1 - 1)); i += blockDim.x) {
      const int t = i & (C - 1), e = i >> lc;
      const int64_t j = (int64_t)e * n2 + t;
      if (j < nv) async_copy(&sm[sm_pos<V>(L, t, e)], zin + j);
      else sm[sm_pos<V>(L, t, e)] = vzero<V>();
    }
    async_wait_all();
    fftr_pass<V, true, true>(0, logn1, C, tw, true, SmAt<V>{sm, L}, SmPut<V>{sm, L});
  } else {
    fftr_pass<V, true, true, true, false, INF>(0, logn1, C, tw, true, [&](int t, int e) {
      const int64_t j = (int64_t)e * n2 + t;
      return j < nv ? zin[j] : vzero<V>();
    }, SmPut<V>{sm, L});
  }
  __syncthreads();
  fftr_passes<V, true, true>(sm, logn1, C, tw, 1, np - 1, false);
  fftr_pass<V, true, true>(np - 1, logn1, C, tw, false, SmAt<V>{sm, L}, [&](int t, int e, const V& v) {
    const int k1 = brev(e, logn1);
    sc[(int64_t)e * n2 + t] = cmul(v, twn[((int64_t)(c0 + t) * k1) & (n - 1)]);
  });
}

// Four-step step B on rows r0 .. r0+rows-1 of the pair's scratch.  spec: the level's
// spectrum (n elements, four-step order).  No barrier at the end.
template <typename T, int INF = 8, bool ASYNC = false>
__device__ __forceinline__ void conv_row_body(Vt<T>* sm, Vt<T>* __restrict__ sc_row, const Vt<T>* __restrict__ spec_all,
                                              int logn1, int logn2, int rows, int r0, const Vt<T>* __restrict__ tw) {
  typedef Vt<T> V;
  const int n2 = 1 << logn2, logn = logn1 + logn2, n = 1 << logn;
  V* __restrict__ sc = sc_row + (int64_t)r0 * n2;
  const V* __restrict__ twn = tw + (n - 2);
  const SmLayout L = sm_layout<V>(logn2);
  const int np = fftr_npasses<V>(logn2);
  if constexpr (ASYNC) {
    for (int i = threadIdx.x; i < (rows << logn2); i += blockDim.x)
      async_copy(&sm[sm_pos<V>(L, i >> logn2, i & (n2 - 1))], sc + i);
    async_wait_all();
    fftr_pass<V, true>(0, logn2, rows, tw, false, SmAt<V>{sm, L}, SmPut<V>{sm, L});
  } else {
    fftr_pass<V, true, false, true, false, INF>(0, logn2, rows, tw, false, [&](int t, int e) { return sc[t * n2 + e]; },
                                                SmPut<V>{sm, L});
  }
  __syncthreads();
  fftr_passes<V, true>(sm, logn2, rows, tw, 1, np - 1, false);
  const V* __restrict__ spec = spec_all + (int64_t)r0 * n2;
  fftr_middle<V>(sm, logn2, rows, [&](int t, int pos0, auto& x, auto RR) {
    SpecMul<V>{spec + t * n2}(t, pos0, x, RR);
  });
  __syncthreads();
  fftr_passes<V, false>(sm, logn2, rows, tw, 1, np - 1, false);
  fftr_pass<V, false>(np - 1, logn2, rows, tw, false, SmAt<V>{sm, L}, [&](int t, int e, const V& v) {
    const int k1 = brev(r0 + t, logn1);
    sc[t * n2 + e] = cmulc(v, twn[((int64_t)e * k1) & (n - 1)]);
  });
}

// Four-step step C on columns c0 .. c0+C-1: inverse column transforms of the scratch,
// result written to the pair's output half zo_row (mode 0: subtracted).  No barrier at
// the end.
template <typename T, int INF = 8, bool ASYNC = false>
__device__ __forceinline__ void conv_col_inv_body(Vt<T>* sm, const Vt<T>* __restrict__ sc_row,
                                                  Vt<T>* __restrict__ zo_row, int logn1, int logn2, int C, int c0,
                                                  int mode, const Vt<T>* __restrict__ tw) {
  typedef Vt<T> V;
  const int n2 = 1 << logn2, h1 = 1 << (logn1 - 1);
  const V* __restrict__ sc = sc_row + c0;
  V* __restrict__ zo = zo_row + c0;
  const SmLayout L = sm_layout<V>(logn1);
  const int np = fftr_npasses<V>(logn1);
  if constexpr (ASYNC) {
    const int lc = 31 - __clz(C);
    for (int i = threadIdx.x; i < (C << logn1); i += blockDim.x) {
      const int t = i & (C - 1), e = i >> lc;
      async_copy(&sm[sm_pos<V>(L, t, e)], sc + (int64_t)e * n2 + t);
    }
    async_wait_all();
    fftr_pass<V, false, true>(0, logn1, C, tw, false, SmAt<V>{sm, L}, SmPut<V>{sm, L});
  } else {
    fftr_pass<V, false, true, true, false, INF>(0, logn1, C, tw, false,
                                                [&](int t, int e) { return sc[(int64_t)e * n2 + t]; }, SmPut<V>{sm, L});
  }
  __syncthreads();
  fftr_passes<V, false, true>(sm, logn1, C, tw, 1, np - 1, false);
  if (mode == 0) {
    fftr_pass<V, false, true, false, true, INF>(np - 1, logn1, C, tw, false, SmAt<V>{sm, L},
                                                SubUpperCols<V>{zo, h1, n2});
  } else {
    fftr_pass<V, false, true>(np - 1, logn1, C, tw, false, SmAt<V>{sm, L}, [&](int t, int e, const V& v) {
      if (e < h1) zo[(int64_t)e * n2 + t] = v;
    });
  }
}

// Split of a four-step length: n1 = 2^(logn/2) columns' length, n2 the rest.
struct Split {
  int logn, logn1, logn2;
};
__host__ __device__ inline Split split_of(int logn) { return Split{logn, logn / 2, logn - logn / 2}; }

// Columns per group of the four-step column steps (power of two): 128-byte row segments,
// at most `cap` elements of shared memory, at most n2.
__host__ __device__ inline int fourstep_cols_for(int logn1, int logn2, int elem_bytes, int cap) {
  int C = 128 / elem_bytes;
  while (C > 2 && ((int64_t)C << logn1) > cap) C >>= 1;
  while (C > 1 && C > (1 << logn2)) C >>= 1;
  return C;
}

}  // namespace
}  // namespace ftoep
