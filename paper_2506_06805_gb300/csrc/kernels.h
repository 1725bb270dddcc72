// Internal kernel entry points (host launchers) of the library.
#pragma once

#include <vector>

#include "common.cuh"

namespace cdfns {

// ---------------------------------------------------------------------------
// Complex GEMM  C(m, n) = alpha * sum_k opA(A)(m, k) * opB(B)(n, k) + beta * C
//
// Operands are addressed through offset tables (element offsets, complex
// units): A(m, k) = A[am[m] + ak[k]], B(n, k) = B[bn[n] + bk[k]],
// C(m, n) = C[cm[m] + cn[n]]. A NULL table means the linear map
// (am[m] = m * lda, ak[k] = k, ... cm[m] = m * ldc, cn[n] = n), so plain
// row-major K-major operands need no table. conj flags conjugate an operand.
// ---------------------------------------------------------------------------
struct GemmDesc {
  long M = 0, N = 0, K = 0;
  const cplx *A = nullptr; const long *am = nullptr, *ak = nullptr; long lda = 0; bool conjA = false;
  const cplx *B = nullptr; const long *bn = nullptr, *bk = nullptr; long ldb = 0; bool conjB = false;
  cplx *C = nullptr; const long *cm = nullptr, *cn = nullptr; long ldc = 0;
  cplx alpha = {1.0, 0.0}, beta = {0.0, 0.0};
  bool k_contig = false;  // the GEMV operand's innermost K index has unit stride
  bool f32 = false;       // GEMV shapes: FP32 products, runs summed in FP64 (tensor-core tiers)
};

// FP64 SIMT path (CC_TIER_FP64).
void gemm_f64(const GemmDesc &g, cudaStream_t st, int num_sms);

// Skinny complex product on the CUDA cores:
//   C[cb(r) + cs(s)] = alpha sum_k G[r][k] S[s][k] + beta C
// for r < Mb (long side), s < Ns (short side), k < K. Row offsets are
// table[i] when the table is given, else i * ld; k offsets gk[k] / sk[k],
// else k * gks / k * sks. G and S are FP64 complex (conjugated on request),
// C is FP64 complex and must not overlap G or S. f64 = false (tensor-core
// tiers, K <= SKINNY_MAX_K): products and sums in FP32, alpha in FP32, beta
// in FP64. f64 = true (K <= SKINNY64_MAX_K): everything in FP64.
constexpr int SKINNY_MAX_K = 48;
constexpr int SKINNY64_MAX_K = 32;
struct SkinnyDesc {
  long Mb = 0;
  int Ns = 0, K = 0;
  const cplx *G = nullptr; const long *gr = nullptr, *gk = nullptr; long ldg = 0, gks = 1;
  bool conjG = false;
  const cplx *S = nullptr; const long *sr = nullptr, *sk = nullptr; long lds = 0, sks = 1;
  bool conjS = false;
  cplx *C = nullptr; const long *cb = nullptr, *cs = nullptr; long ldcb = 0, ldcs = 0;
  cplx alpha = {1.0, 0.0}, beta = {0.0, 0.0};
  bool f64 = false;
};
void gemm_skinny(const SkinnyDesc &d, cudaStream_t st);

// Real tensor-core GEMM on the expanded complex form (tcgen05, TMEM, TMA).
//   D(r, n) = sum_k A'(r, k) B'(n, k),  r < Mr = 2 M, k < Kp (padded)
// A' rows 2m / 2m+1 hold (Re, -Im) / (Im, Re) of A(m, :) interleaved over k,
// B' row n holds (Re, Im) of B(n, :), so rows 2m, 2m+1 of D are Re, Im of
// (A B^T)(m, n). Planes are fp32 (tf32 kinds) or bf16, row-major with
// leading dimension Kp; *_lo planes hold the low parts for the 3-product
// split tiers (NULL otherwise).
enum TcOut {
  TC_OUT_F64 = 0,        // C(m, n) = alpha D + beta C through tables (double2)
  TC_OUT_F64_ATOMIC = 1, // C(m, n) += alpha D (split-K partials)
  TC_OUT_F32 = 2,        // Cf[m * ldc + n] = D (float2, plain row-major)
};
struct TcDesc {
  long M = 0, N = 0, Kp = 0;  // complex rows, columns, padded real K
  const void *A = nullptr, *Alo = nullptr, *B = nullptr, *Blo = nullptr;
  int tier = TIER_TF32;
  int out = TC_OUT_F64;
  void *C = nullptr; const long *cm = nullptr, *cn = nullptr; long ldc = 0;
  cplx alpha = {1.0, 0.0}, beta = {0.0, 0.0};
  int split_k = 1;
  // tile choices (0 = automatic): output tile width 128 or 256, m-tiles per
  // raster group, K blocks per TMEM promotion chunk
  int bn = 0, group_m = 0, chunk = 0;
  // TIER_FP16: device floats holding max |element| of A and of B; the planes
  // were packed with fp16_scale() of these and the product is unscaled in
  // the epilogue (nullptr: unscaled)
  const float *amax_a = nullptr, *amax_b = nullptr;
  // TC_OUT_F32, or TC_OUT_F64 with beta = 0: atomically raised to amax_mul
  // x max |Re|, |Im| (in FP32) over the values written (the caller zeroes
  // it); nullptr: not tracked
  float *amax_out = nullptr;
  float amax_mul = 1.0f;
  // never time tile candidates for this call (the autotuner allocates a
  // scratch output and events): use a cached choice or the defaults
  bool no_tune = false;
};
void gemm_tc(const TcDesc &g, cudaStream_t st, int *err_flag);
// Several independent GEMMs (any shapes, same or mixed tiers) in as few
// persistent launches as possible: one per tier and tile width, up to 16
// problems each, sharing one tile queue.
void gemm_tc_grouped(const std::vector<TcDesc> &descs, cudaStream_t st, int *err_flag);
// Padded K granularity (real elements) for a tier: 32 for tf32, 64 for bf16.
// Tile width for N columns: 256 unless 128-wide tiles waste clearly less
// to padding.
int tc_pick_bn(long N);
// K split count for a GEMM of `tiles` output tiles and nkb K blocks: the
// count (<= 32, >= 4 K blocks per split) that best fills whole waves of
// num_sms persistent CTAs, slightly favouring fewer splits; 1 when the
// tiles already make 8 or more waves.
int tc_pick_split(long tiles, long nkb, int num_sms);
int tc_k_align(int tier);
// Limit of every pipeline wait in the tensor-core kernels launched from now
// on (ns; 0 restores the default of 2 s). Waits that drain copies and MMAs
// before a kernel exits keep their own 2 s limit.
void tc_set_wait_limit(unsigned long long ns);
unsigned long long tc_wait_limit();
size_t tc_elem_bytes(int tier);

// Expand/convert operands for gemm_tc from FP64 tensors addressed by tables.
// A side: rows 2m, 2m+1 (M complex rows) x Kp real columns (2 per complex k).
// TIER_FP16: amax (device float, from tc_absmax) sets the operand's scale.
// rows_unit: neighbouring rows are (mostly) neighbouring elements while k
// is strided; the operand is then read along rows and transposed through
// shared memory.
void tc_pack_A(const cplx *src, const long *am, const long *ak, long lda,
               bool conj, long M, long K, long Kp, int tier, void *hi,
               void *lo, cudaStream_t st, const float *amax = nullptr, bool rows_unit = false);
void tc_pack_B(const cplx *src, const long *bn, const long *bk, long ldb,
               bool conj, long N, long K, long Kp, int tier, void *hi,
               void *lo, cudaStream_t st, const float *amax = nullptr, bool rows_unit = false);
// *amax = max over the operand's elements of max(|Re|, |Im|), addressed like
// tc_pack_A / tc_pack_B (rows x K through tables or strides).
void tc_absmax(const cplx *src, const long *rt, const long *kt, long ld, long rows, long K,
               float *amax, cudaStream_t st);

// ---------------------------------------------------------------------------
// Tensor helpers
// ---------------------------------------------------------------------------
// table[i] = sum_d digit_d(i) * stride_d over the row-major index space dims.
void make_offsets(long *table, int nd, const long *dims, const long *strides,
                  cudaStream_t st);
// C(m, n) *= beta through tables (or linear when NULL).
void scale_2d(cplx *C, const long *cm, const long *cn, long ldc, long M,
              long N, cplx beta, cudaStream_t st);
// y = alpha * x + beta * y (contiguous)
void axpby(long n, cplx alpha, const cplx *x, cplx beta, cplx *y,
           cudaStream_t st);
// out[perm-ordered] = alpha * in + beta * out, generic rank <= 8 permutation:
// out element with row-major index over odims reads in[sum digit * istr].
void permute(cplx *out, const cplx *in, int nd, const long *odims,
             const long *istr, cplx alpha, cplx beta, bool conj,
             cudaStream_t st);

// R += c (X - s_ij X(ji) - s_ab X(ba) + s_ij s_ab X(ji,ba)) on [o][o][v][v]
// tensors, mode bit 0 = P(ij), bit 1 = P(ab); tiled through shared memory.
void antisym_add(cplx *R, const cplx *X, int o, int v, double c, int mode, cudaStream_t st);

// Deterministic FP64 reductions (two-pass, fixed order).
// sum_i w * conj?(x_i) * y_i
cplx dot(const cplx *x, const cplx *y, long n, bool conj_x, cudaStream_t st,
         cplx *dev_scratch /* >= 1024 */, cplx *host_out = nullptr);
// Same, result left on the device (no synchronisation).
// Counts, over x[0..n), the values whose integer-pipe narrowing differs
// from __double2float_rn (bad[0]) and whose widening of that FP32 value
// differs from the hardware conversion (bad[1]); bad is 2 device counters.
void conversion_check(const double *x, long n, unsigned long long *bad, cudaStream_t st);
// res[k * res_stride] = sum_i conj(xs[k][i]) y[i] for k < m <= 16, one pass
// over y; f32: FP32 products and per-thread sums (block sums in FP64).
// scratch: at least m device cplx, more for more blocks.
void dot_multi(const cplx *const *xs, int m, const cplx *y, long n, bool f32, cplx *res,
               long res_stride, cplx *scratch, long scratch_len, cudaStream_t st);
void dot_dev(const cplx *x, const cplx *y, long n, bool conj_x, cplx *res,
             cudaStream_t st, cplx *dev_scratch);

// Single-step pivoted Cholesky decomposition (Eq. 21) of M = B B^H, B
// [N][r] on the device: vectors L [n][N] (n <= max_vec, row-major), pivots
// piv[n] on the host (may be NULL); returns n.
int pivoted_cholesky(const cplx *B, long N, int r, double tau, int max_vec, cplx *L, long *piv,
                     Allocator *al, cudaStream_t st, int num_sms);

}  // namespace cdfns
