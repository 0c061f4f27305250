// Register-radix FFT engine on shared memory (Sec. 3.1: every Toeplitz product is a
// circulant one, C = F^-1 diag(F c) F).
//
// Same transforms as fft_dif / fft_dit in fft.cuh -- forward decimation in frequency
// (natural order in, bit-reversed order out) and the mirrored inverse decimation in time
// (bit-reversed in, natural out, unnormalised) -- computed in passes that each merge
// r = log2(R) radix-2 stages: a thread loads R elements at stride m = g/R of one group of
// size g, runs the r stages in registers, and stores them back in place.  One pass of
// radix 8 replaces three shared-memory round trips and three barriers of the stage-by-stage
// form (the engine supports radix up to 16); the in-place order of a merged pass is exactly that of its stages, so outputs,
// spectra and partner indices keep the bit-reversed convention.
//
// Twiddles: stage k of a pass (sub-group size G = g/2^k) multiplies element (i + j m) by
// W_G^(i + jl m) = W_G^i * W_{2h}^jl, h = R/2^(k+1), jl = j mod 2h.  W_G^i is one table
// load per stage (table W_n^k at offset n-2); W_{2h}^jl is a compile-time constant
// (1, -i and (+-1-i)/sqrt2 are done without multiplications).  In a pass with m = 1 every
// W_G^i is 1 and no table is read.
//
// Shared-memory layout: `cnt` transforms of length n = 2^logn back to back; element e of
// transform t sits at  t*n + (e ^ (((e >> RB) ^ brev(t)) & xm)),  RB = log2(pass radix),
// xm = min(n, 2^S) - 1 with S = log2(elements per 128-byte wavefront), brev over
// log2(xm+1) bits.  The XOR only changes the low S bits (a permutation inside each
// 2^S-element chunk, invertible because its source bits start at RB); with the source
// shifted by the pass radix every pass of the schedule below, the column-wise (one lane per
// transform) loads and stores and natural-order access are free of bank conflicts (checked
// exhaustively with a bank model for 8- and 16-byte elements at radix 8 and 16).
#pragma once

#include "fft.cuh"

namespace ftoep {

template <int V_>
struct IntC {
  static constexpr int value = V_;
};
template <int B, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(IntC<B>{});
    static_for<B + 1, E>(f);
  }
}

template <typename V> struct EngineTraits;
template <> struct EngineTraits<float2> {
  static constexpr int S = 4;   // 16 elements of 8 bytes per wavefront
  // radix-8 passes: radix 16 needs one pass fewer but ~40 more registers per thread; the
  // float kernels are latency-bound, and the extra resident warps of radix 8 were worth more
  // (measured on the batched solve: 3.04 s against 3.11 s per step)
  static constexpr int RB = 3;
};
template <> struct EngineTraits<double2> {
  static constexpr int S = 3;
  static constexpr int RB = 3;  // radix-8 passes
};
template <> struct EngineTraits<ff2> {
  static constexpr int S = 3;
  static constexpr int RB = 3;
};

struct SmLayout {
  int logn;
  int lb;  // log2(xm + 1)
  int xm;
};

template <typename V>
__device__ __forceinline__ SmLayout sm_layout(int logn) {
  constexpr int S = EngineTraits<V>::S;
  SmLayout L;
  L.logn = logn;
  L.lb = logn < S ? logn : S;
  L.xm = (1 << L.lb) - 1;
  return L;
}

template <typename V>
__device__ __forceinline__ int sm_pos(const SmLayout& L, int t, int e) {
  constexpr int RB = EngineTraits<V>::RB;
  const int bt = L.lb ? (int)(__brev((unsigned)(t & L.xm)) >> (32 - L.lb)) : 0;
  return (t << L.logn) + (e ^ (((e >> RB) ^ bt) & L.xm));
}

// ------------------------------------------------------------------ constant twiddles

// cos(pi/8), sin(pi/8)
constexpr double kC8 = 0.92387953251128675613;
constexpr double kS8 = 0.38268343236508977173;
constexpr double kR2 = 0.70710678118654752440;  // sqrt(1/2)

__device__ __forceinline__ float2 vconst(float2, double x, double y) { return make_float2((float)x, (float)y); }
__device__ __forceinline__ double2 vconst(double2, double x, double y) { return make_double2(x, y); }
__device__ __forceinline__ ff2 vconst(ff2, double x, double y) {
  ff2 r;
  r.xh = (float)x;
  r.xl = (float)(x - (double)(float)x);
  r.yh = (float)y;
  r.yl = (float)(y - (double)(float)y);
  return r;
}

// Constant factors are applied with their rounding error folded back in (float: the
// constant as hi + lo, products formed with FMAs), so every product is rounded once.
// Without this the float constants carry the same relative error into every element they
// touch -- a bias that adds up coherently across a transform and across the levels of
// the solve instead of averaging out like independent roundings.
__host__ __device__ constexpr float fhi(double c) { return (float)c; }
__host__ __device__ constexpr float flo(double c) { return (float)(c - (double)(float)c); }

__device__ __forceinline__ double2 scale_r2(double2 v) { return make_double2(v.x * kR2, v.y * kR2); }
__device__ __forceinline__ float2 scale_r2(float2 v) {
  constexpr float h = fhi(kR2), l = flo(kR2);
  return make_float2(fmaf(v.x, h, v.x * l), fmaf(v.y, h, v.y * l));
}
__device__ __forceinline__ ff2 scale_r2(ff2 v) {
  const float h = (float)kR2, l = (float)(kR2 - (double)(float)kR2);
  ff2 r;
  ff_mul(v.xh, v.xl, h, l, r.xh, r.xl);
  ff_mul(v.yh, v.yl, h, l, r.yh, r.yl);
  return r;
}

// v * W_8 = v (1 - i)/sqrt2 = ((x + y) + i (y - x))/sqrt2
template <typename V> __device__ __forceinline__ V mul_w8(V v) {
  V r;
  r.x = v.x + v.y;
  r.y = v.y - v.x;
  return scale_r2(r);
}
// v * W_8^3 = v (-1 - i)/sqrt2 = ((y - x) - i (x + y))/sqrt2
template <typename V> __device__ __forceinline__ V mul_w83(V v) {
  V r;
  r.x = v.y - v.x;
  r.y = -(v.x + v.y);
  return scale_r2(r);
}
// v * conj(W_8) = v (1 + i)/sqrt2 = ((x - y) + i (x + y))/sqrt2
template <typename V> __device__ __forceinline__ V mul_w8c(V v) {
  V r;
  r.x = v.x - v.y;
  r.y = v.x + v.y;
  return scale_r2(r);
}
// v * conj(W_8^3) = v (-1 + i)/sqrt2 = (-(x + y) + i (x - y))/sqrt2
template <typename V> __device__ __forceinline__ V mul_w83c(V v) {
  V r;
  r.x = -(v.x + v.y);
  r.y = v.x - v.y;
  return scale_r2(r);
}
template <> __device__ __forceinline__ ff2 mul_w8<ff2>(ff2 v) {
  ff2 r;
  ff_add_fast(v.xh, v.xl, v.yh, v.yl, r.xh, r.xl);
  ff_add_fast(v.yh, v.yl, -v.xh, -v.xl, r.yh, r.yl);
  return scale_r2(r);
}
template <> __device__ __forceinline__ ff2 mul_w83<ff2>(ff2 v) {
  ff2 r;
  ff_add_fast(v.yh, v.yl, -v.xh, -v.xl, r.xh, r.xl);
  ff_add_fast(-v.xh, -v.xl, -v.yh, -v.yl, r.yh, r.yl);
  return scale_r2(r);
}
template <> __device__ __forceinline__ ff2 mul_w8c<ff2>(ff2 v) {
  ff2 r;
  ff_add_fast(v.xh, v.xl, -v.yh, -v.yl, r.xh, r.xl);
  ff_add_fast(v.xh, v.xl, v.yh, v.yl, r.yh, r.yl);
  return scale_r2(r);
}
template <> __device__ __forceinline__ ff2 mul_w83c<ff2>(ff2 v) {
  ff2 r;
  ff_add_fast(-v.xh, -v.xl, -v.yh, -v.yl, r.xh, r.xl);
  ff_add_fast(v.xh, v.xl, -v.yh, -v.yl, r.yh, r.yl);
  return scale_r2(r);
}

// W_16^J for odd J: (re, im)
template <int J>
struct W16 {
  static constexpr double re = J == 1 ? kC8 : J == 3 ? kS8 : J == 5 ? -kS8 : -kC8;
  static constexpr double im = J == 1 ? -kS8 : J == 3 ? -kC8 : J == 5 ? -kC8 : -kS8;
};
template <typename V, int J>
__device__ __forceinline__ V w16() {
  return vconst(V{}, W16<J>::re, W16<J>::im);
}
// v * W_16^J (conj: v * conj(W_16^J)); float: constant as hi + lo
template <int J, bool CONJ>
__device__ __forceinline__ float2 mul_w16(float2 v) {
  constexpr float ah = fhi(W16<J>::re), al = flo(W16<J>::re);
  constexpr float bh = fhi(CONJ ? -W16<J>::im : W16<J>::im), bl = flo(CONJ ? -W16<J>::im : W16<J>::im);
  float2 r;
  r.x = fmaf(v.x, ah, fmaf(-v.y, bh, fmaf(v.x, al, -v.y * bl)));
  r.y = fmaf(v.x, bh, fmaf(v.y, ah, fmaf(v.x, bl, v.y * al)));
  return r;
}
template <int J, bool CONJ>
__device__ __forceinline__ double2 mul_w16(double2 v) {
  return CONJ ? cmulc(v, w16<double2, J>()) : cmul(v, w16<double2, J>());
}
template <int J, bool CONJ>
__device__ __forceinline__ ff2 mul_w16(ff2 v) {
  return CONJ ? cmulc(v, w16<ff2, J>()) : cmul(v, w16<ff2, J>());
}

// v * W_N2^J (0 <= J < N2/2, N2 in {2, 4, 8, 16})
template <typename V, int N2, int J>
__device__ __forceinline__ V mul_wc(V v) {
  if constexpr (J == 0) {
    return v;
  } else if constexpr (4 * J == N2) {
    return mul_mi(v);
  } else if constexpr (8 * J == N2) {
    return mul_w8(v);
  } else if constexpr (8 * J == 3 * N2) {
    return mul_w83(v);
  } else {
    static_assert(N2 == 16, "constant twiddles up to radix 16");
    return mul_w16<J, false>(v);
  }
}
// v * conj(W_N2^J)
template <typename V, int N2, int J>
__device__ __forceinline__ V mul_wcc(V v) {
  if constexpr (J == 0) {
    return v;
  } else if constexpr (4 * J == N2) {
    return mul_pi(v);
  } else if constexpr (8 * J == N2) {
    return mul_w8c(v);
  } else if constexpr (8 * J == 3 * N2) {
    return mul_w83c(v);
  } else {
    static_assert(N2 == 16, "constant twiddles up to radix 16");
    return mul_w16<J, true>(v);
  }
}

// ------------------------------------------------------------------ register passes

// Forward: x[j] = element i + j m of a group of size g = 2^logg (m = g / 2^r).
// HZ: x[j] = 0 for j >= 2^(r-1) (not read).  TW: apply the table twiddles (m > 1).
template <typename V, int r, bool HZ, bool TW>
__device__ __forceinline__ void dif_regs(V (&x)[1 << r], const V* __restrict__ tw, int logg, int i) {
  constexpr int R = 1 << r;
  static_for<0, r>([&](auto KK) {
    constexpr int k = decltype(KK)::value;
    constexpr int half = R >> (k + 1);
    [[maybe_unused]] V w;
    if constexpr (TW) w = tw[(1 << (logg - k)) - 2 + i];
    static_for<0, R>([&](auto JJ) {
      constexpr int j = decltype(JJ)::value;
      if constexpr ((j & half) == 0) {
        constexpr int jl = j & (2 * half - 1);
        const V u = x[j];
        V d;
        if constexpr (HZ && k == 0) {
          d = u;
        } else {
          const V v = x[j + half];
          x[j] = cadd(u, v);
          d = csub(u, v);
        }
        d = mul_wc<V, 2 * half, jl>(d);
        if constexpr (TW) d = cmul(d, w);
        x[j + half] = d;
      }
    });
  });
}

// Inverse (mirror of dif_regs): stages from the smallest sub-group to the largest.
template <typename V, int r, bool TW>
__device__ __forceinline__ void dit_regs(V (&x)[1 << r], const V* __restrict__ tw, int logg, int i) {
  constexpr int R = 1 << r;
  static_for<0, r>([&](auto KK) {
    constexpr int k = r - 1 - decltype(KK)::value;
    constexpr int half = R >> (k + 1);
    [[maybe_unused]] V w;
    if constexpr (TW) w = tw[(1 << (logg - k)) - 2 + i];
    static_for<0, R>([&](auto JJ) {
      constexpr int j = decltype(JJ)::value;
      if constexpr ((j & half) == 0) {
        constexpr int jl = j & (2 * half - 1);
        V v = x[j + half];
        if constexpr (TW) v = cmulc(v, w);
        v = mul_wcc<V, 2 * half, jl>(v);
        const V u = x[j];
        x[j] = cadd(u, v);
        x[j + half] = csub(u, v);
      }
    });
  });
}

// ------------------------------------------------------------------ pass schedule

// DIF passes p = 0..np-1: pass 0 has radix 2^r0 on groups of size n, every later pass
// radix 2^RB; the last one works on groups of size 2^RB (m = 1).  DIT runs the mirror:
// DIT pass q is DIF pass np-1-q.
struct FftPlan {
  int logn, np, r0, rb;
  // log2 of the group size of DIF pass p
  __device__ __forceinline__ int logg(int p) const { return p == 0 ? logn : logn - r0 - (p - 1) * rb; }
};

template <typename V>
__device__ __forceinline__ FftPlan fft_plan(int logn) {
  constexpr int RB = EngineTraits<V>::RB;
  FftPlan P;
  P.logn = logn;
  P.rb = RB;
  P.r0 = logn % RB;
  if (P.r0 == 0) P.r0 = RB;
  if (logn == 0) P.r0 = 0;
  P.np = logn == 0 ? 0 : 1 + (logn - P.r0) / RB;
  return P;
}

// One pass over all units: Ld(t, e) -> V, St(t, e, V).  DIF or DIT, radix 2^r.
// HZ (DIF only): inputs j >= R/2 are zero and Ld is not called for them.
// TM (transform-major): consecutive threads take consecutive transforms (cnt a power of
// two) -- the mapping for column transforms whose global loads are coalesced across
// transforms; otherwise consecutive threads take consecutive units of one transform.
template <typename V, int r, bool DIF, bool HZ, bool TM, int UB, bool RMW, class Ld, class St>
__device__ __forceinline__ void run_pass(int logn, int cnt, int logg, const V* __restrict__ tw, Ld ld, St st) {
  constexpr int R = 1 << r;
  const int lm = logg - r;
  const int lu = logn - r;
  const int tot = cnt << lu;
  // UB units per thread per iteration: all their loads (and, for a read-modify-write
  // storer, the fetches of the values it updates) are issued before any arithmetic, which
  // keeps UB*R global loads in flight
  for (int u0 = threadIdx.x; u0 < tot; u0 += blockDim.x * UB) {
    V x[UB][R];
    [[maybe_unused]] V f[RMW ? UB : 1][RMW ? R : 1];
    int tq[UB], e0q[UB], iq[UB];
    static_for<0, UB>([&](auto QQ) {
      constexpr int q = decltype(QQ)::value;
      const int u = u0 + q * (int)blockDim.x;
      int t, b;
      if constexpr (TM) {
        t = u & (cnt - 1);
        b = u / cnt;
      } else {
        t = u >> lu;
        b = u & ((1 << lu) - 1);
      }
      const int grp = b >> lm;
      iq[q] = b & ((1 << lm) - 1);
      tq[q] = t;
      e0q[q] = (grp << logg) + iq[q];
      if (UB == 1 || u < tot) {
        static_for<0, R>([&](auto JJ) {
          constexpr int j = decltype(JJ)::value;
          if constexpr (HZ && j >= R / 2) {
            x[q][j] = vzero<V>();
          } else {
            x[q][j] = ld(t, e0q[q] + (j << lm));
          }
          if constexpr (RMW) f[q][j] = st.fetch(t, e0q[q] + (j << lm));
        });
      }
    });
    static_for<0, UB>([&](auto QQ) {
      constexpr int q = decltype(QQ)::value;
      if (UB == 1 || u0 + q * (int)blockDim.x < tot) {
        if (lm == 0) {
          if constexpr (DIF) dif_regs<V, r, HZ, false>(x[q], tw, logg, 0);
          else dit_regs<V, r, false>(x[q], tw, logg, 0);
        } else {
          if constexpr (DIF) dif_regs<V, r, HZ, true>(x[q], tw, logg, iq[q]);
          else dit_regs<V, r, true>(x[q], tw, logg, iq[q]);
        }
        static_for<0, R>([&](auto JJ) {
          constexpr int j = decltype(JJ)::value;
          if constexpr (RMW) st(tq[q], e0q[q] + (j << lm), x[q][j], f[q][j]);
          else st(tq[q], e0q[q] + (j << lm), x[q][j]);
        });
      }
    });
  }
}

// Pass p of the schedule (DIF pass p, or DIT pass p = DIF pass np-1-p) with the given
// loader and storer.  No barrier.
// GL: the loader reads global memory (several units per thread keep loads in flight).
// RMW: the storer updates global memory: st.fetch(t, e) is called in the load phase and
// st(t, e, v, fetched) after the arithmetic.
// INF: elements a thread keeps in flight in a global-memory pass (units per thread = INF / radix).
template <typename V, bool DIF, bool TM = false, bool GL = false, bool RMW = false, int INF = 8, class Ld, class St>
__device__ __forceinline__ void fftr_pass(int p, int logn, int cnt, const V* __restrict__ tw, bool half_zero, Ld ld,
                                          St st) {
  constexpr int RB = EngineTraits<V>::RB;
  const FftPlan P = fft_plan<V>(logn);
  const int pd = DIF ? p : P.np - 1 - p;
  const int r = pd == 0 ? P.r0 : P.rb;
  const int logg = P.logg(pd);
  const bool hz = DIF && pd == 0 && half_zero;
#define FTOEP_PASS_CASE(RR)                                                                     \
  {                                                                                             \
    constexpr int LH = (1 << RR) / 2, LF = 1 << RR;                                             \
    constexpr int UBH = (GL || RMW) ? (LH >= INF ? 1 : INF / LH) : 1;                           \
    constexpr int UBF = (GL || RMW) ? (LF >= INF ? 1 : INF / LF) : 1;                           \
    if (hz) run_pass<V, RR, DIF, true, TM, UBH, RMW>(logn, cnt, logg, tw, ld, st);              \
    else run_pass<V, RR, DIF, false, TM, UBF, RMW>(logn, cnt, logg, tw, ld, st);                \
  }
  switch (r) {
    case 1: { FTOEP_PASS_CASE(1) break; }
    case 2: { FTOEP_PASS_CASE(2) break; }
    case 3: { FTOEP_PASS_CASE(3) break; }
    default:
      if constexpr (RB >= 4) { FTOEP_PASS_CASE(4) }
      break;
  }
#undef FTOEP_PASS_CASE
}

// ------------------------------------------------------------------ drivers

// Shared-memory accessors for the layout above.
template <typename V>
struct SmAt {
  const V* a;
  SmLayout L;
  __device__ __forceinline__ V operator()(int t, int e) const { return a[sm_pos<V>(L, t, e)]; }
};
template <typename V>
struct SmPut {
  V* a;
  SmLayout L;
  __device__ __forceinline__ void operator()(int t, int e, const V& v) const { a[sm_pos<V>(L, t, e)] = v; }
};

template <typename V>
__device__ __forceinline__ int fftr_npasses(int logn) {
  return fft_plan<V>(logn).np;
}

// Passes [p0, p1) in shared memory (DIF or DIT numbering), a barrier after each.
template <typename V, bool DIF, bool TM = false>
__device__ void fftr_passes(V* a, int logn, int cnt, const V* __restrict__ tw, int p0, int p1, bool half_zero) {
  const int np = fftr_npasses<V>(logn);
  const SmLayout L = sm_layout<V>(logn);
  for (int p = p0; p < p1 && p < np; ++p) {
    fftr_pass<V, DIF, TM>(p, logn, cnt, tw, half_zero, SmAt<V>{a, L}, SmPut<V>{a, L});
    __syncthreads();
  }
}

// Whole transforms in shared memory; the caller has stored the input with sm_pos.
template <typename V, bool TM = false>
__device__ void fftr_dif(V* a, int logn, int cnt, const V* __restrict__ tw, bool half_zero) {
  fftr_passes<V, true, TM>(a, logn, cnt, tw, 0, 1 << 20, half_zero);
}
template <typename V, bool TM = false>
__device__ void fftr_dit(V* a, int logn, int cnt, const V* __restrict__ tw) {
  fftr_passes<V, false, TM>(a, logn, cnt, tw, 0, 1 << 20, false);
}

// The last DIF pass, a pointwise operation on the spectrum, and the first DIT pass, fused
// in registers (groups of size 2^r, m = 1, no table twiddles).  op(t, pos0, x, IntC<R>)
// receives the spectrum values at storage positions pos0 .. pos0 + R - 1 (bit-reversed
// frequency order) of transform t and modifies them in place.  No barrier.
template <typename V, int r, class Op>
__device__ __forceinline__ void middle_r(V* a, int logn, int cnt, Op op) {
  constexpr int R = 1 << r;
  const SmLayout L = sm_layout<V>(logn);
  const int lu = logn - r;
  const int tot = cnt << lu;
  for (int u = threadIdx.x; u < tot; u += blockDim.x) {
    const int t = u >> lu, grp = u & ((1 << lu) - 1);
    const int e0 = grp << r;
    V x[R];
    static_for<0, R>([&](auto JJ) {
      constexpr int j = decltype(JJ)::value;
      x[j] = a[sm_pos<V>(L, t, e0 + j)];
    });
    dif_regs<V, r, false, false>(x, nullptr, r, 0);
    op(t, e0, x, IntC<R>{});
    dit_regs<V, r, false>(x, nullptr, r, 0);
    static_for<0, R>([&](auto JJ) {
      constexpr int j = decltype(JJ)::value;
      a[sm_pos<V>(L, t, e0 + j)] = x[j];
    });
  }
}

// Runs DIF pass np-1 + op + DIT pass 0.
template <typename V, class Op>
__device__ __forceinline__ void fftr_middle(V* a, int logn, int cnt, Op op) {
  const FftPlan P = fft_plan<V>(logn);
  const int r = P.np == 1 ? P.r0 : P.rb;
  switch (r) {
    case 1: middle_r<V, 1>(a, logn, cnt, op); break;
    case 2: middle_r<V, 2>(a, logn, cnt, op); break;
    case 3: middle_r<V, 3>(a, logn, cnt, op); break;
    default:
      if constexpr (EngineTraits<V>::RB >= 4) middle_r<V, 4>(a, logn, cnt, op);
      break;
  }
}

// Storage-order partner inside group 0 of the last pass: the frequency at position j of the
// group is brev_r(j) * n/R, its partner n - that (mod n).
__host__ __device__ constexpr int brev_c(int x, int bits) { return bits == 0 ? 0 : ((x & 1) << (bits - 1)) | brev_c(x >> 1, bits - 1); }
__host__ __device__ constexpr int group0_partner(int j, int r) { return brev_c(((1 << r) - brev_c(j, r)) & ((1 << r) - 1), r); }

// As fftr_middle, for a pointwise operation that pairs each frequency k with its partner
// n - k.  Group g of the last pass (storage positions g R .. g R + R - 1, frequencies
// brev(position)) pairs with group g ^ (2^h - 1), h its highest set bit, element j with
// element R-1-j; groups 0 and 1 pair with themselves (group 0 by group0_partner, group 1
// j with R-1-j).  Item u of a transform takes groups 0 and 1 (u = 0) or the pair with
// g = u + 2^floor(log2 u), so consecutive threads read consecutive groups.
// pair(t, pa, pb, wa, wb) gets the values at storage positions pa and pb (partners) and
// replaces both; self(t, p, w) a self-partner frequency (0 or n/2).  No barrier.
template <typename V, int r, class Pair, class Self>
__device__ __forceinline__ void middle_partner_r(V* a, int logn, int cnt, Pair pair, Self self) {
  constexpr int R = 1 << r;
  const SmLayout L = sm_layout<V>(logn);
  const int lu = logn - r;  // >= 1
  const int lh = lu - 1;
  for (int w = threadIdx.x; w < (cnt << lh); w += blockDim.x) {
    const int t = w >> lh, u = w & ((1 << lh) - 1);
    int g = 0, gp = 1;
    if (u > 0) {
      const int hb1 = 31 - __clz(u);
      g = u + (1 << hb1);
      gp = g ^ ((2 << hb1) - 1);
    }
    V xa[R], xb[R];
    static_for<0, R>([&](auto JJ) {
      constexpr int j = decltype(JJ)::value;
      xa[j] = a[sm_pos<V>(L, t, (g << r) + j)];
      xb[j] = a[sm_pos<V>(L, t, (gp << r) + j)];
    });
    dif_regs<V, r, false, false>(xa, nullptr, r, 0);
    dif_regs<V, r, false, false>(xb, nullptr, r, 0);
    if (u == 0) {
      static_for<0, R>([&](auto JJ) {
        constexpr int j = decltype(JJ)::value;
        constexpr int jp = group0_partner(j, r);
        if constexpr (jp == j) self(t, j, xa[j]);
        else if constexpr (j < jp) pair(t, j, jp, xa[j], xa[jp]);
      });
      static_for<0, R / 2>([&](auto JJ) {
        constexpr int j = decltype(JJ)::value;
        pair(t, R + j, 2 * R - 1 - j, xb[j], xb[R - 1 - j]);
      });
    } else {
      static_for<0, R>([&](auto JJ) {
        constexpr int j = decltype(JJ)::value;
        pair(t, (g << r) + j, (gp << r) + R - 1 - j, xa[j], xb[R - 1 - j]);
      });
    }
    dit_regs<V, r, false>(xa, nullptr, r, 0);
    dit_regs<V, r, false>(xb, nullptr, r, 0);
    static_for<0, R>([&](auto JJ) {
      constexpr int j = decltype(JJ)::value;
      a[sm_pos<V>(L, t, (g << r) + j)] = xa[j];
      a[sm_pos<V>(L, t, (gp << r) + j)] = xb[j];
    });
  }
}

// Runs DIF pass np-1 + the partner-paired operation + DIT pass 0 (np >= 2).
template <typename V, class Pair, class Self>
__device__ __forceinline__ void fftr_middle_partner(V* a, int logn, int cnt, Pair pair, Self self) {
  middle_partner_r<V, EngineTraits<V>::RB>(a, logn, cnt, pair, self);  // the last pass has radix RB
}

}  // namespace ftoep
