// Elementwise and packing kernels of the CCSD / IP-EOM path.
#pragma once

#include "common.cuh"

namespace cdfns {

// --- input staging -----------------------------------------------------------
// Split one chunk of L^P (P in [p0, p0+np), [np][n][n]) into the oo/ov/vo/vv
// blocks ([X][o][o] ...), and accumulate validation maxima into stats
// (double bits, atomicMax): [0] max |L|, [1] max |L_pq - conj(L_qp)|,
// [2] non-finite count.
void split_cholesky(const cplx *chunk, int np, int p0, int o, int v, cplx *Loo, cplx *Lov,
                    cplx *Lvo, cplx *Lvv, unsigned long long *stats, cudaStream_t st);

// --- amplitudes ----------------------------------------------------------------
// out[ijab] = t2[ijab] + f * (t1[ia] t1[jb] - t1[ib] t1[ja])
// fp32_t1: form the t1 t1 part in FP32 (tensor-core tiers only)
// mx (optional, three device floats): set to max(|Re|, |Im|) in FP32 over
// [0] t2, [1] the first output, [2] the second output (0 when absent), the
// FP16 tiers' operand scale sources, found in the same pass
void make_tau(const cplx *t1, const cplx *t2, cplx *out, int o, int v, double f,
              cudaStream_t st, bool fp32_t1 = false, float *mx = nullptr);
// tau (f = 1) and tau~ (f = 1/2) in one pass over t2
void make_tau_pair(const cplx *t1, const cplx *t2, cplx *tau, cplx *taut, int o, int v,
                   cudaStream_t st, bool fp32_t1 = false, float *mx = nullptr);
// t_new = R / D with D from eps (FP64); exact zeros on i=j or a=b.
void jacobi(const cplx *R1, const cplx *R2, const double *eps, int o, int v, cplx *t1,
            cplx *t2, cudaStream_t st);
// MP2 start: t2 = conj(oovv) / D2, t1 = 0.
void mp2_amplitudes(const cplx *oovv, const double *eps, int o, int v, cplx *t1, cplx *t2,
                    cudaStream_t st);
// Unique amplitudes: [t1 (o*v)] + [t2 i<j, a<b (row-major pairs)].
void pack_amps(const cplx *t1, const cplx *t2, int o, int v, const int *ij_i, const int *ij_j,
               const int *ab_a, const int *ab_b, cplx *vec, cudaStream_t st);
void unpack_amps(const cplx *vec, int o, int v, cplx *t1, cplx *t2, cudaStream_t st);
// inv[k] = 1 / D_k for the packed amplitudes (FP64)
void amp_denoms(const double *eps, int o, int v, const int *ij_i, const int *ij_j, const int *ab_a,
                const int *ab_b, double *inv, cudaStream_t st);
// vec = packed(R) * inv (the Jacobi step, unique amplitudes only)
void jacobi_packed(const cplx *R1, const cplx *R2, const double *inv, int o, int v, const int *ij_i,
                   const int *ij_j, const int *ab_a, const int *ab_b, cplx *vec, cudaStream_t st);
long energy_scratch_len(int o, int v);
// *res = sum_{i<j,a<b} <ij||ab> (t_ij^ab + t_i^a t_j^b - t_i^b t_j^a) from a
// packed vector (the CCSD energy, Eq. 15); scratch holds block partials.
void energy_packed(const cplx *oovv, const cplx *vec, int o, int v, const int *ij_i,
                   const int *ij_j, const int *ab_a, const int *ab_b, bool f32, cplx *scratch,
                   long scratch_len, cplx *res, cudaStream_t st);
// Weighted squared norm helpers are done with dot() on packed vectors.

// --- DIIS ------------------------------------------------------------------------
// Solve the (m+1) Pulay system with Hermitian B (m x m, row-major, device)
// in FP64 by Gaussian elimination with partial pivoting; coef[m] receives
// the weights; status[0] = 0 ok, 1 singular.
void diis_solve(const cplx *B, int m, int ldb, cplx *coef, int *status, cudaStream_t st);
// out = sum_i coef[i] * vecs[i] (m <= 16 vectors)
void diis_combine(cplx *const *vecs, const cplx *coef, int m, long n, cplx *out,
                  cudaStream_t st);

// --- ladder ------------------------------------------------------------------------
// Antisymmetrise one V slab into the packed B operand of the second GEMM:
// W[(a,b)][(c<d)] = V[a][c][b][d] - V[a][d][b][c] for the a<b pairs
// p in [p0, p1) (global row-major pair order). V is [nA*v][(v-a0)*v]
// complex (float2 if f32 else double2), rows (a - a0, c), cols (b - a0, d).
// Output: fp32 planes (re, im interleaved over k, row stride kp, hi + lo),
// bf16 planes, or a double2 matrix [p1-p0][ncd].
// FP16 tiers: fp16 plane(s) scaled by fp16_scale(*amax), amax a bound on
// |W| (twice the slab maximum recorded by the GEMM that wrote V).
void ladder_antisym(const void *V, bool f32, int v, int a0, int nA, long p0, long p1,
                    const int *pair_a, const int *pair_b, const int *cd_c, const int *cd_d,
                    int tier, void *hi, void *lo, long kp, cplx *w64, cudaStream_t st,
                    const float *amax = nullptr);

// MP2 amplitudes of the pairs (i, j) with j = i + 1 + j', j' < nj, from
// G[j'][a][b] = sum_P L^P_ai L^P_bj: t[j'][a][b] = (G[j'][a][b] - G[j'][b][a])
// / (eps_i + eps_j - eps_a - eps_b) (= <ab||ij> / D, Eqs. 23-24).
void mp2_pair_amplitudes(const cplx *G, const double *eps, int o, int v, int i, int nj, cplx *t,
                         cudaStream_t st);

// R2[i][j][a][b] += R[(i<j)][(a<b)] with the four antisymmetric images.
void unpack_pairs_add(const cplx *R, int o, int v, const int *ij_i, const int *ij_j,
                      const int *ab_a, const int *ab_b, cplx *R2, cudaStream_t st);
// Pair tables (row-major i<j order).
void make_pairs(int n, int *pi, int *pj, cudaStream_t st);

// --- IP vectors --------------------------------------------------------------------
// packed [k][o + npair*v] <-> r1 [k][o], r2 [k][o][o][v] (antisymmetric)
void ip_unpack(const cplx *vec, int k, int o, int v, cplx *r1, cplx *r2, cudaStream_t st);
void ip_pack(const cplx *r1, const cplx *r2, int k, int o, int v, cplx *vec, cudaStream_t st);
// d[o + pairs*v]: -Hoo_ii and Hvv_bb - Hoo_ii - Hoo_jj
void ip_diag(const cplx *Hoo, const cplx *Hvv, int o, int v, cplx *d, cudaStream_t st);
// s2[K][i][j][b] += (dvv_b - doo_i - doo_j) r2, s1[K][i] -= doo_i r1 (the
// diagonal one-body part of sigma, exact in FP64)
void ip_diag_apply(const cplx *r1, const cplx *r2, const cplx *doo, const cplx *dvv, int k, int o,
                   int v, cplx *s1, cplx *s2, cudaStream_t st);
// s2 += tA + tB + tC - (X1 - X1(i<->j)) + (X2 - X2(i<->j)), [k][o][o][v]
void sigma_combine(cplx *s2, const cplx *tA, const cplx *tB, const cplx *tC, const cplx *X1,
                   const cplx *X2, int k, int o, int v, cudaStream_t st);
// off = A with zero diagonal, diag = diagonal of A (n x n)
void split_diag(const cplx *A, int n, cplx *off, cplx *diag, cudaStream_t st);
// x[r] = R[r] / (w[r] - d) with |den| floored at 1e-8
void precondition(const cplx *R, const cplx *w, const cplx *d, int nr, long dim, cplx *x,
                  cudaStream_t st);
// x[r] *= 1/norm[r] (norm from device array of complex dots (re part))
void scale_rows_inv_sqrt(cplx *x, const cplx *dots, int nr, long dim, cudaStream_t st);

// --- misc ----------------------------------------------------------------------------
// A[i][i] += diag[i] (square n x n, row-major)
void add_diag(cplx *A, const double *diag, int n, cudaStream_t st);
// out[k] = |x[k]|^2 weight-summed by block is done by dot(); this fills NaN check.
// Bit-exact Eq. 23 block dump: out[p][q][r][s] = sum_P (L_pr L_qs - L_ps L_qr),
// P ascending, no FMA. Blocks address L through per-index spaces.
void dump_block(const cplx *Lpr, long spr_P, long spr_p, long spr_r, const cplx *Lqs,
                long sqs_P, long sqs_q, long sqs_s, const cplx *Lps, long sps_P, long sps_p,
                long sps_s, const cplx *Lqr, long sqr_P, long sqr_q, long sqr_r, int X, int np,
                int nq, int nr, int ns, cplx *out, cudaStream_t st);

}  // namespace cdfns
