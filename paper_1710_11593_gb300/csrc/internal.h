// Internal interfaces between the host orchestration (api.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace ftoep {

// ---------------------------------------------------------------- host math (weights.cpp)
double digamma(double x);
double scheme_scale(int kind, double gamma, double tau);
// a[j] (j < n) and optionally da/dgamma; see weights.cpp for the formulas.
void scheme_weights(int kind, double gamma, double tau, int64_t n, double* a, double* dadg);
// right-hand-side weights of u0 and phi at levels 1..n
void initial_weights(int kind, double gamma, double tau, int64_t n, double* wu0, double* wphi);
// first column e_j (j < n) of the time operator acting on v_k = (u^k - u^{k-1})/tau
void difference_weights(int kind, double gamma, double tau, int64_t n, double* e);

// Twiddle tables W_n^k for n = 2 .. maxtw (powers of two) at offset n-2, host side
// (api.cu); any output may be NULL.
void host_twiddles(int64_t maxtw, std::vector<double2>* h64, std::vector<float2>* h32, std::vector<float4>* hff);
// Message for ftoep_last_error(NULL, ...) (api.cu).
void set_global_error(const char* msg);

// ---------------------------------------------------------------- kernel launchers
// Storage precision of the complex work arrays: 0 = double2, 1 = float2,
// 2 = float-float pairs (ff2, products of the mixed path's residual).
enum Prec { P64 = 0, P32 = 1, PFF = 2 };

struct DstArgs {
  // forward: f (+ wu0*u0 + wphi*phi) [M][N] doubles (or f32)  ->  z pairs [P][ld]
  // inverse: z pairs -> u [M][N] doubles (write or accumulate) or u32 floats
  // Pair p holds modes p+1 (.x) and M-p (.y) (space 1) or rows 2p, 2p+1 (space 0).
  const double* f;      // forward input
  const float* f32;     // forward input in float instead of f (no initial-data terms)
  float* u32;           // inverse output in float instead of u (write only)
  double dst_scale;     // 1/sqrt(2K)
  const double* u0;     // nullable
  const double* phi;    // nullable
  const double* wu0;    // length N (with u0)
  const double* wphi;   // length N (with phi)
  double* u;            // inverse output
  void* z;              // pair array (double2 or float2)
  int64_t ld;           // row length of z (elements)
  int64_t N;            // valid time columns
  int64_t ncols;        // columns to process (>= N; columns >= N are written as 0 by forward)
  int64_t M;            // interior points
  int logK2;            // log2(2(M+1))
  int reverse;          // time reversal of z (forward: write z[N-1-n]; inverse: read z[N-1-n])
  int accumulate;       // inverse: u += result
  int space;            // 0: no transform (pairs of rows), 1: sine transform
  int diff_form;        // forward: right-hand side of the difference form (-(S u0) instead of wu0*u0)
  // Sine transform for M+1 not a power of two, a DFT of length L by Bluestein as a cyclic
  // convolution of length P = 2^logP >= 2L - 1.  Double: the folded half-length form (L = K,
  // the real DFT of y_j = s_j (x_j + x_{K-j}) + (x_j - x_{K-j})/2, s_j = sin(pi j/K)); float:
  // the odd extension (L = 2K).
  int bluestein;
  int K;                // M + 1
  int logP;
  const void* chirp;    // c_n = exp(-i pi n^2 / L), n < L (z precision)
  const void* bspec;    // forward transform (this library's order) of conj(chirp) wrapped to length P, / P
  const void* sinv;     // double: s_j = sin(pi j / K), j = 0 .. K/2
  double inv_h2;        // 1/h^2 (space 1) for S u0
  double lambda;        // lambda (space 0) for S u0
  const void* tw;       // twiddles of the z precision
};
int launch_dst_forward(Prec prec, const DstArgs& a, cudaStream_t st);
// Largest M+1 the Bluestein sine transform handles in one block's shared memory.
int bluestein_max_K(Prec prec);
int launch_dst_inverse(Prec prec, const DstArgs& a, cudaStream_t st);

// Pack real lines [nlines][N] into pairs [ceil(nlines/2)][ld] (zero padded to ld, optional
// reversal within [0,N)); unpack back.
struct PackArgs {
  const double* x;  // lines (pack input)
  const float* x32; // lines in float instead of x
  double* y;        // lines (unpack output)
  void* z;          // pairs
  int64_t ld, N, nlines;
  int reverse;
  int mode;  // unpack: 0 write, 1 accumulate
};
int launch_pack(Prec prec, const PackArgs& a, cudaStream_t st);
int launch_unpack(Prec prec, const PackArgs& a, cudaStream_t st);

// Time prefix sums along every line of [M][N] doubles, in double precision:
//   reverse = 0: out[j][n] = base + tau * sum_{k<=n} in[j][k], base = out[j][n] (accumulate)
//                or u0[j] (u0 != NULL) or 0;
//   reverse = 1: out[j][n] = tau * sum_{k>=n} in[j][k].
// in may equal out.
// in32 (float input, forward only): the sums are float-float; tau = tau_h + tau_l.
struct ScanArgs {
  const double* in;
  const float* in32;
  float tau_h, tau_l;
  double* out;
  const double* u0;
  int64_t N, M;
  double tau;
  int accumulate;
  int reverse;
};
int launch_scan(const ScanArgs& a, cudaStream_t st);

// Residual r = f + wu0*u0 + wphi*phi - (T x) - S(u) in float, with (T x) given in
// float-float pairs (line 2p in .x, 2p+1 in .y) and S the spatial operator: Dirichlet
// -u_xx (space 1) or lambda*u (space 0).
struct ResidualArgs {
  const double* f;
  const double* u0;
  const double* phi;
  const double* wu0;
  const double* wphi;
  const double* u;
  const void* tu;     // ff2 pairs [ceil(M/2)][ld]
  float* r32;
  int64_t ld, N, M;
  int space;
  double inv_h2, lambda;
  int cn;                // Crank-Nicolson: S acts on (u^n + u^{n-1})/2
  const double* uprev0;  // with cn: u0, the level before the first (NULL = zero)
};
int launch_residual(const ResidualArgs& a, cudaStream_t st);

// Sum over all (line, n) of x[line][n] * tu_pair(line, n)  ->  partial sums per block.
struct DotArgs {
  const double* x;    // lines [nlines][N]
  const double2* tu;  // pairs
  int64_t ld, N, nlines;
  double* partial;    // [gridDim]
  int nblocks;
};
int launch_dot(const DotArgs& a, cudaStream_t st);
int launch_sum(const double* partial, int n, double* out, cudaStream_t st);

// Kernel spectrum of c_k = (lo <= k < hi) ? a[k] : 0, k < n = 2^logn, computed in double
// and stored (divided by n) in the order of the convolution path chosen for n:
// shared-memory DIF if n <= nsmem, else the four-step split n = n1*n2.
struct SpecArgs {
  const double* a;
  int64_t lo, hi;
  int logn;
  int nsmem;
  void* out;               // length n, precision of the convolution
  const double2* tw64;     // double twiddles
  double2* scratch64;      // length n (four-step only)
};
int launch_spectrum(Prec prec, const SpecArgs& a, cudaStream_t st);

// Circulant convolution of every pair row:  t = x (*) c over length n = 2^logn, where
// x = z_in[p][in_off .. in_off + n/2) zero-padded.  mode 0 (half-split update):
// z_out[p][out_off + i] -= t[n/2 + i];  mode 1 (product): z_out[p][out_off + i] = t[i];
// both for i < n/2.
struct ConvArgs {
  void* zin;
  void* zout;
  int64_t ld_in, ld_out, in_off, out_off;
  int64_t npairs;
  int logn;
  int nsmem;
  int mode;
  const void* spec;
  const void* tw;
  void* scratch;    // [npairs][n] (four-step only)
  int64_t nvalid;   // four-step step A: input entries at index >= nvalid read as zero (0: none)
};
int launch_conv(Prec prec, const ConvArgs& a, cudaStream_t st);
// One column step of the four-step convolution alone (length n = 2^logn > nsmem):
// inverse = 0: step A (zin -> scratch), 1: step C (scratch -> zout, mode as above).
int launch_fourstep_cols(Prec prec, const ConvArgs& a, int inverse, cudaStream_t st);

// Inverse-series solve of every pair: x = h * y over the padded length Np, as one cyclic
// convolution of length n = 2 Np (exact for the first Np outputs) with the pair's packed
// inverse spectrum -- two modes with different kernels in one complex FFT, so the
// spectrum product pairs each frequency with its partner n - k (as the block inverse).
// Four-step only (n above the shared-memory convolution length).
struct FinvArgs {
  void* z;           // pairs [npairs][ld]: right-hand side in, solution out (first Np entries)
  int64_t ld;
  int64_t N;         // right-hand side entries; entries N .. Np-1 are read as zero
  int64_t npairs;
  int logn;          // n = 2 Np
  const void* cs;    // packed spectra [npairs][n], four-step storage order, scaled by 1/n
  const void* tw;
  void* scratch;     // [npairs][n]
};
int launch_full_inverse(Prec prec, const FinvArgs& a, cudaStream_t st);

// Plan time: the packed spectra of the pairs' inverse columns h (double, first Np entries
// of each pair row; zero-padded to n = 2 Np) in precision prec.
struct FinvSpecArgs {
  const double2* h;  // [npairs][ld]
  int64_t ld;
  int64_t N;         // entries of h used (the rest read as zero)
  int64_t npairs;
  int logn;
  double2* scratch64;  // [npairs][n]
  void* cs;            // [npairs][n]
  const double2* tw64;
};
int launch_finv_spectrum(Prec prec, const FinvSpecArgs& a, cudaStream_t st);

// Restarted GMRES vector kernels (gmres.cu), fields [M][N] double, L = M N.
constexpr int kMaxBasis = 64;  // largest restart length
int launch_space_add(double* y, const double* x, int64_t M, int64_t N, int space, double inv_h2, double lambda,
                     double sw, cudaStream_t st);
// partial[i * nblocks + b] = block b's part of <V_i, w>, i < k (V_i = V + i * ldv)
int launch_mdot(const double* V, int64_t ldv, int k, const double* w, int64_t L, double* partial, int nblocks,
                cudaStream_t st);
// w += sum_{i<k} c_i V_i (c: k doubles in device memory, k <= kMaxBasis)
int launch_maxpy(double* w, const double* V, int64_t ldv, int k, const double* c, int64_t L, cudaStream_t st);
// all nodes of a sweep: g[i][n] = c F[i][n] + s0[i] w0[n] + s1[i] w1[n] (w0/s0, w1/s1 nullable)
int launch_sweep_rhs_lines(double* g, const double* F, const double* w0, const double* s0, const double* w1,
                           const double* s1, int64_t M, int64_t N, double c, cudaStream_t st);
// out[i] = in[i] + t[i - d] (i >= d), in[i] below; lines of N doubles
int launch_shift_add_lines(double* out, const double* in, const double* t, int64_t M, int64_t N, int64_t d,
                           cudaStream_t st);
// y = a x + b z (z unread when b = 0)
int launch_lincomb(double* y, double a, const double* x, double b, const double* z, int64_t L, cudaStream_t st);

// Solve the lower-triangular Toeplitz systems of every pair on one time block
// [t0, t0 + B) in place (history from earlier blocks already subtracted).
struct BlockArgs {
  void* z;
  int64_t ld;
  int64_t npairs;
  int64_t t0;
  int B;            // block length (power of two)
  int L;            // leaf length (power of two <= 16, <= B)
  int Sf;           // first FFT level (levels L <= s < Sf are dense products)
  const double* a;  // e[0..B): shared first column (difference form)
  const double2* invdiag;  // per pair: 1/(e0 + lambda*tau) of its two modes
  const double2* lamtau;   // per pair: lambda*tau of its two modes (all-ones part of the operator)
  double2* prefix;         // per pair: running sums of the solved v (in: before t0, out: after)
  const void* spec;        // spectra of levels Sf..B/2 (level s at offset 2(s - Sf))
  const void* tw;
};
int launch_block_solve(Prec prec, const BlockArgs& a, cudaStream_t st);
size_t block_solve_smem(Prec prec, int B, int Sf);

// Block solve by the inverse of the block operator (block_inverse.cu): per pair the
// spectra C1, C2 (length 2B, this library's FFT order, divided by 2B) of the two modes'
// inverse first columns h (first B entries of T_m^-1 e_1), Hermitian-packed into one
// length-2B array c1 (C1 at the lower of two partner positions, C2 at the other; c2 unused).
struct InvSpecArgs {
  const double2* h;   // [npairs][ldh]: h of the pair's first mode in .x, of its second mode in .y
  int64_t ldh;
  int64_t npairs;
  int B, logB;
  void* c1;           // [npairs][2B], precision of the solve
  void* c2;
  const double2* tw64;
};
int launch_inverse_spectrum(Prec prec, const InvSpecArgs& a, cudaStream_t st);
int launch_unit_impulse(double2* z, int64_t ld, int64_t npairs, int B, cudaStream_t st);

struct BlockInvArgs {
  void* z;                 // pairs [npairs][ld]; block [t0, t0+B) in place
  int64_t ld, npairs, t0;
  int B, logB;
  const void* c1;
  const void* c2;
  const double2* lamtau;   // per pair lambda*tau
  double2* prefix;         // per pair running sums of the solved v (in and out)
  const void* tw;
};
int launch_block_inverse(Prec prec, const BlockInvArgs& a, cudaStream_t st);

// Persistent per-pair solve (chain.cu): one launch runs the whole time recursion (block
// solves and every cross-block level) of every listed pair, one pair per block at a time.
struct ChainProb {
  void* z;                 // pairs [P][ld] of the problem, precision of the launch
  int64_t ld;
  const void* c1;          // packed block-inverse spectra [P][2B]
  const double2* lamtau;   // per pair lambda*tau
  const void* spec;        // level spectra (level s at offset 2(s - Sf))
  int64_t Sf;
  int nblk, logB;
};
struct ChainArgs {
  const ChainProb* probs;
  const int2* items;        // (index into probs, pair), longest chains first
  int nitems;
  unsigned* counter;        // next item; zero at launch
  void* scratch;            // four-step scratch, scratch_per_block elements per block
  int64_t scratch_per_block;
  int smem_elems;           // dynamic shared memory in elements of the launch precision
  int nsmem;                // largest shared-memory convolution length (nsmem_for)
  const void* tw;
};
// Dynamic shared memory of the chain kernel for block lengths up to maxB.
size_t chain_smem_bytes(Prec prec, int maxB);
// Resident blocks per SM of the chain kernel with that shared memory (0 on failure).
int chain_blocks_per_sm(Prec prec, size_t smem);
int launch_chain(Prec prec, const ChainArgs& a, int grid, size_t smem, cudaStream_t st);

// Largest shared-memory FFT length of each precision.
int nsmem_for(Prec prec);
// Opt a kernel in to `bytes` of dynamic shared memory (once per kernel and size).
void set_smem_once(const void* fn, size_t bytes);

}  // namespace ftoep
