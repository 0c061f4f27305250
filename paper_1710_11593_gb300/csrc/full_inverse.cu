// Inverse-series solve of the per-mode lower-triangular Toeplitz systems: each mode's
// operator T_m (difference form, E + lambda_m tau (1 - (1 - sw) I)) has a lower-triangular
// Toeplitz inverse whose first column h_m = T_m^-1 e_1 is the power series of the inverse
// symbol.  With h_m known over the whole padded length Np, a solve is one causal
// convolution x = h_m * y -- the O(N log N) per-mode alternative to the recursive half
// split of Sec. 3 (whose levels cost O(N log^2 N)); the products are circulant ones
// (Sec. 3.1, Eq. be1) of length n = 2 Np, exact for the first Np outputs.
//
// Two modes share one complex FFT (pair p: modes in .x and .y), with different real
// kernels, so the spectrum product pairs frequency k with its partner n - k:
//     Y_k = C1_k Z_k + C2_k conj(Z_{n-k}),  C1 = (H_a + H_b)/2,  C2 = (H_a - H_b)/2.
// Four-step layout (n = n1 n2, steps A and C are the level convolutions' column kernels):
// scratch row r holds k1 = brev(r) and position q of a row holds k2 = brev(q), k = k1 + n1 k2.
// The partner of (r, q) is (0, partner_pos(q)) in row 0 (k1 = 0), else row r' with
// brev(r') = n1 - brev(r) at position n2 - 1 - q.  So row 0 and row 1 (k1 = n1/2) pair with
// themselves and every other row with one partner row; the row kernel keeps partner rows
// together in one block's shared memory.  The packed spectrum stores C1 at the lower of the
// two partner storage indices and C2 at the higher (the self-partner frequencies 0 and
// n/2, both in row 0, hold the real pair (C1, C2) in one slot).
#include <type_traits>

#include "block_inverse_body.cuh"
#include "internal.h"

namespace ftoep {

namespace {

constexpr int kThreads = 256;

inline void set_smem(const void* fn, size_t bytes) { set_smem_once(fn, bytes); }

template <typename V>
__device__ __forceinline__ V conjv(V a) {
  a.y = -a.y;
  return a;
}

// Rows of block b: block 0 the two self-partner rows 0 and 1; block b >= 1 the row pairs
// (brev(u), brev(n1 - u)) of u = u0 .. u0 + units - 1 (slot 2g: brev(u), slot 2g+1: its
// partner), u0 = 1 + (b - 1) G.
struct RowSet {
  int b, u0, units, logn1, n1;
  __device__ __forceinline__ int row(int t) const {
    if (b == 0) return t;
    const int u = u0 + (t >> 1);
    return brev((t & 1) ? (n1 - u) : u, logn1);
  }
  __device__ __forceinline__ int slots() const { return b == 0 ? 2 : 2 * units; }
};

__device__ __forceinline__ RowSet row_set(int b, int logn1, int G) {
  RowSet R;
  R.b = b;
  R.logn1 = logn1;
  R.n1 = 1 << logn1;
  R.u0 = 1 + (b - 1) * G;
  R.units = b == 0 ? 1 : min(G, R.n1 / 2 - R.u0);
  return R;
}

// Partner product on the transformed rows in shared memory (storage order of the forward
// row transforms).  Every frequency pair is visited once.
template <typename V>
__device__ __forceinline__ void partner_product(V* sm, const SmLayout& L, const RowSet& R, int logn2,
                                                const V* __restrict__ cs) {
  const int n2 = 1 << logn2;
  if (R.b == 0) {
    for (int qq = threadIdx.x; qq < 2 * n2; qq += blockDim.x) {
      const int t = qq >> logn2, pos = qq & (n2 - 1);
      const int pp = t == 0 ? partner_pos(pos, logn2) : n2 - 1 - pos;
      if (pp < pos) continue;
      const int q1 = sm_pos<V>(L, t, pos);
      const V z1 = sm[q1];
      const V* c = cs + (int64_t)t * n2;
      if (pp == pos) {  // self partner: real C1, C2 in one slot
        const V cc = c[pos];
        V r;
        r.x = cc.x * z1.x + cc.y * z1.x;
        r.y = cc.x * z1.y - cc.y * z1.y;
        sm[q1] = r;
      } else {
        const V c1 = c[pos], c2 = c[pp];
        const int q2 = sm_pos<V>(L, t, pp);
        const V z2 = sm[q2];
        sm[q1] = cadd(cmul(c1, z1), cmul(c2, conjv(z2)));
        sm[q2] = cadd(cmulc(z2, c1), cmulc(conjv(z1), c2));
      }
    }
    return;
  }
  for (int qq = threadIdx.x; qq < (R.units << logn2); qq += blockDim.x) {
    const int g = qq >> logn2, pos = qq & (n2 - 1);
    const int ta = 2 * g, tb = 2 * g + 1;
    const int posb = n2 - 1 - pos;
    const int64_t ia = (int64_t)R.row(ta) * n2 + pos, ib = (int64_t)R.row(tb) * n2 + posb;
    const bool alow = ia < ib;
    const V c1 = cs[alow ? ia : ib], c2 = cs[alow ? ib : ia];
    const int qa = sm_pos<V>(L, ta, pos), qb = sm_pos<V>(L, tb, posb);
    const int ql = alow ? qa : qb, qh = alow ? qb : qa;
    const V z1 = sm[ql], z2 = sm[qh];
    sm[ql] = cadd(cmul(c1, z1), cmul(c2, conjv(z2)));
    sm[qh] = cadd(cmulc(z2, c1), cmulc(conjv(z1), c2));
  }
}

// Four-step step B of the inverse-series solve: the rows of one RowSet of one pair --
// forward row transforms, partner product with the pair's packed spectrum, inverse row
// transforms, the four-step twiddle removed -- in place in the pair's scratch.
template <typename T>
__global__ void __launch_bounds__(kThreads) finv_row_kernel(FinvArgs A, int logn1, int logn2, int G) {
  typedef Vt<T> V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int n2 = 1 << logn2, logn = logn1 + logn2;
  const int64_t n = (int64_t)1 << logn;
  const int64_t p = blockIdx.y;
  V* __restrict__ sc = (V*)A.scratch + p * n;
  const V* __restrict__ cs = (const V*)A.cs + p * n;
  const V* __restrict__ tw = (const V*)A.tw;
  const V* __restrict__ twn = tw + (n - 2);
  const RowSet R = row_set(blockIdx.x, logn1, G);
  const int cnt = R.slots();
  const SmLayout L = sm_layout<V>(logn2);
  const int np = fftr_npasses<V>(logn2);
  fftr_pass<V, true, false, true, false, 8>(0, logn2, cnt, tw, false,
                                            [&](int t, int e) { return sc[(int64_t)R.row(t) * n2 + e]; },
                                            SmPut<V>{sm, L});
  __syncthreads();
  fftr_passes<V, true>(sm, logn2, cnt, tw, 1, np, false);
  partner_product<V>(sm, L, R, logn2, cs);
  __syncthreads();
  fftr_passes<V, false>(sm, logn2, cnt, tw, 0, np - 1, false);
  fftr_pass<V, false>(np - 1, logn2, cnt, tw, false, SmAt<V>{sm, L}, [&](int t, int e, const V& v) {
    const int r = R.row(t);
    const int k1 = brev(r, logn1);
    sc[(int64_t)r * n2 + e] = cmulc(v, twn[((int64_t)e * k1) & (n - 1)]);
  });
}

// Plan time, after step A on h: forward row transforms of every row of every pair, in
// place (double), `rows` rows per block.
__global__ void __launch_bounds__(kThreads) finv_rowfft_kernel(FinvSpecArgs A, int logn1, int logn2, int rows) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double2* sm = reinterpret_cast<double2*>(smraw);
  const int n2 = 1 << logn2;
  const int64_t n = (int64_t)n2 << logn1;
  double2* sc = A.scratch64 + (int64_t)blockIdx.y * n + (int64_t)blockIdx.x * rows * n2;
  const SmLayout L = sm_layout<double2>(logn2);
  fftr_pass<double2, true, false, true, false, 8>(0, logn2, rows, A.tw64, false,
                                                  [&](int t, int e) { return sc[(int64_t)t * n2 + e]; },
                                                  SmPut<double2>{sm, L});
  __syncthreads();
  fftr_passes<double2, true>(sm, logn2, rows, A.tw64, 1, 1 << 20, false);
  for (int i = threadIdx.x; i < (rows << logn2); i += blockDim.x) {
    const int t = i >> logn2, e = i & (n2 - 1);
    sc[(int64_t)t * n2 + e] = sm[sm_pos<double2>(L, t, e)];
  }
}

template <typename V>
__device__ __forceinline__ V from_d2(double x, double y) {
  V r;
  r.x = x;
  r.y = y;
  return r;
}

// Plan time: packed C1/C2 of every pair from H = FFT_n(h_a + i h_b) in four-step storage:
// H_a(k) = (H_k + conj H_{n-k})/2, H_b(k) = (H_k - conj H_{n-k})/(2i), scaled by 1/n.
template <typename T>
__global__ void __launch_bounds__(kThreads) finv_pack_kernel(FinvSpecArgs A, int logn1, int logn2) {
  typedef Vt<T> V;
  const int n1 = 1 << logn1, n2 = 1 << logn2;
  const int64_t n = (int64_t)n1 * n2;
  const int64_t p = blockIdx.y;
  const double2* H = A.scratch64 + p * n;
  V* cs = (V*)A.cs + p * n;
  const double inv = 1.0 / (double)n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(i >> logn2), pos = (int)(i & (n2 - 1));
    const int k1 = brev(r, logn1);
    int64_t j;
    if (k1 == 0) {
      j = partner_pos(pos, logn2);
    } else {
      j = (int64_t)brev(n1 - k1, logn1) * n2 + (n2 - 1 - pos);
    }
    if (j < i) continue;
    const double2 hk = H[i], hm = H[j];
    // H_a = (hk + conj hm)/2, H_b = (hk - conj hm)/(2i)
    const double ar = 0.5 * (hk.x + hm.x), ai = 0.5 * (hk.y - hm.y);
    const double br = 0.5 * (hk.y + hm.y), bi = -0.5 * (hk.x - hm.x);
    const double c1r = 0.5 * (ar + br) * inv, c1i = 0.5 * (ai + bi) * inv;
    const double c2r = 0.5 * (ar - br) * inv, c2i = 0.5 * (ai - bi) * inv;
    if (j == i) {
      cs[i] = from_d2<V>(c1r, c2r);
    } else {
      cs[i] = from_d2<V>(c1r, c1i);
      cs[j] = from_d2<V>(c2r, c2i);
    }
  }
}

// Row pairs per block of the solve's row kernel: about 2048 elements per block.
int finv_units(int logn2) {
  int G = 2048 >> (logn2 + 1);
  return G < 1 ? 1 : G;
}

template <typename T>
void full_inverse_launch(const FinvArgs& a, cudaStream_t st) {
  ConvArgs ca{};
  ca.zin = a.z;
  ca.zout = a.z;
  ca.ld_in = ca.ld_out = a.ld;
  ca.in_off = ca.out_off = 0;
  ca.npairs = a.npairs;
  ca.logn = a.logn;
  ca.mode = 1;
  ca.tw = a.tw;
  ca.scratch = a.scratch;
  ca.nvalid = a.N;
  launch_fourstep_cols(std::is_same<T, double>::value ? P64 : P32, ca, 0, st);
  Split sp = split_of(a.logn);
  const int G = finv_units(sp.logn2);
  const int n1 = 1 << sp.logn1;
  const unsigned nb = 1u + (unsigned)((n1 / 2 - 1 + G - 1) / G);
  const size_t smem = (size_t)2 * G * ((size_t)1 << sp.logn2) * sizeof(Vt<T>);
  set_smem((const void*)finv_row_kernel<T>, smem);
  finv_row_kernel<T><<<dim3(nb, (unsigned)a.npairs), kThreads, smem, st>>>(a, sp.logn1, sp.logn2, G);
  launch_fourstep_cols(std::is_same<T, double>::value ? P64 : P32, ca, 1, st);
}

}  // namespace

int launch_full_inverse(Prec prec, const FinvArgs& a, cudaStream_t st) {
  if (prec == P64) full_inverse_launch<double>(a, st);
  else full_inverse_launch<float>(a, st);
  return 3;
}

int launch_finv_spectrum(Prec prec, const FinvSpecArgs& a, cudaStream_t st) {
  ConvArgs ca{};
  ca.zin = (void*)a.h;
  ca.ld_in = a.ld;
  ca.npairs = a.npairs;
  ca.logn = a.logn;
  ca.tw = a.tw64;
  ca.scratch = a.scratch64;
  ca.nvalid = a.N;
  launch_fourstep_cols(P64, ca, 0, st);
  Split sp = split_of(a.logn);
  int rows = 2048 >> sp.logn2;
  if (rows < 1) rows = 1;
  const size_t smem = (size_t)rows * ((size_t)1 << sp.logn2) * sizeof(double2);
  set_smem((const void*)finv_rowfft_kernel, smem);
  finv_rowfft_kernel<<<dim3((unsigned)((1 << sp.logn1) / rows), (unsigned)a.npairs), kThreads, smem, st>>>(
      a, sp.logn1, sp.logn2, rows);
  const int64_t n = (int64_t)1 << a.logn;
  const unsigned gx = (unsigned)std::min<int64_t>((n + kThreads - 1) / kThreads, 1024);
  if (prec == P64) finv_pack_kernel<double><<<dim3(gx, (unsigned)a.npairs), kThreads, 0, st>>>(a, sp.logn1, sp.logn2);
  else finv_pack_kernel<float><<<dim3(gx, (unsigned)a.npairs), kThreads, 0, st>>>(a, sp.logn1, sp.logn2);
  return 3;
}

}  // namespace ftoep
