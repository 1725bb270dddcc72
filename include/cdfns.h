/*
 * cdfns.h -- C ABI of the GB300 CD/FNS IP-EOM-CCSD library (libcdfns.so).
 *
 * The library computes ionisation potentials with the equation-of-motion
 * coupled-cluster method at the singles-and-doubles level (IP-EOM-CCSD,
 * Eqs. 16-18) on top of CCSD (Eqs. 12-15), with two-electron integrals
 * assembled from complex Cholesky vectors (Eqs. 21-23) and an optional
 * frozen-natural-spinor truncation of the virtual space (Eqs. 24-28).
 * Every contraction runs in CUDA kernels of this library on one GPU.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Return value: CC_OK (0) or a negative CC_ERR_* code. After an error,
 *   cc_last_error() returns a one-line message. A call that fails with
 *   CC_ERR_ARG, CC_ERR_INPUT or CC_ERR_STATE leaves the context unchanged.
 * - Complex numbers are interleaved (re, im) doubles ("complex128").
 * - Spinor index p in [0, n), n = n_occ + n_virt, occupied spinors first.
 *   All arrays are row-major (C order).
 * - Units: Hartree. IPs are positive: omega = E(N-1) - E(N) (Eq. 18).
 * - Ownership: inputs are copied; the library keeps no caller pointer and
 *   writes only to the output arguments of the call. Host pointers are
 *   named *_host or documented as host; *_dev pointers are device memory
 *   on the context's device.
 * - Call order: cc_init -> [fns_truncate] -> ccsd_solve -> ipeom_solve.
 * - Streams: work is issued on the context's stream (cc_set_stream); calls
 *   that return host results synchronise that stream before returning.
 */
#ifndef CDFNS_H
#define CDFNS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CC_OK 0
#define CC_ERR_ARG (-1)           /* bad argument (size, pointer, range) */
#define CC_ERR_INPUT (-2)         /* input data invalid: NaN/Inf, non-Hermitian L */
#define CC_ERR_OOM (-3)           /* device allocation failed */
#define CC_ERR_CUDA (-4)          /* CUDA runtime/driver error */
#define CC_ERR_NOT_CONVERGED (-5) /* iteration limit reached; results written */
#define CC_ERR_NUMERIC (-6)       /* NaN/Inf appeared during the iterations */
#define CC_ERR_TIMEOUT (-7)       /* a bounded device wait gave up */
#define CC_ERR_STATE (-8)         /* call made out of order */
#define CC_ERR_UNSUPPORTED (-9)   /* feature not available on this device */

/* Precision tiers of the contractions (cc_set_precision). Control steps
 * (denominators, DIIS, energies, norms, Davidson subspace) are FP64 in
 * every tier. */
#define CC_TIER_FP64 0   /* complex FP64 on the FP64 pipe (plain path) */
#define CC_TIER_TF32 1   /* tcgen05 kind::tf32, one pass, FP32 accumulate */
#define CC_TIER_TF32X3 2 /* tcgen05 tf32, hi/lo split, 3 products */
#define CC_TIER_BF16X3 3 /* tcgen05 kind::f16 bf16, hi/lo split, 3 products */
#define CC_TIER_FP16 4   /* tcgen05 kind::f16 fp16, one pass, FP32 accumulate;
                          * each operand scaled by a power of two chosen from
                          * its largest magnitude, so the product rounding is
                          * that of TF32 (11-bit significands) at twice the
                          * tensor-core rate */
#define CC_TIER_FP16X3 5 /* kind::f16 fp16 hi/lo split of the scaled operands,
                          * 3 products: TF32X3-class accuracy at the f16 rate */

typedef struct cc_ctx cc_ctx; /* one molecular (synthetic) system */

/* Process-wide defaults picked up by contexts created afterwards.
 * alloc(bytes, user) must return device memory aligned to 256 bytes or NULL;
 * free(ptr, user) releases it. Pass NULLs to restore cudaMalloc/cudaFree.
 * During one library call, a context without a memory limit keeps the
 * blocks it releases and hands them to its next requests of the same size;
 * it frees whatever it still keeps before the call returns (and at once,
 * then retries, when an allocation fails).
 * stream is a cudaStream_t (NULL = legacy default stream). */
int cc_set_default_allocator(void *(*alloc)(size_t, void *),
                             void (*free_fn)(void *, void *), void *user);
int cc_set_default_stream(void *stream);
/* Allocator of one context from now on (same contract as the default; NULLs
 * restore cudaMalloc/cudaFree). Buffers the context already holds are
 * released later through the functions that allocated them. Errors:
 * CC_ERR_ARG (NULL ctx, or only one of alloc/free given). */
int cc_set_allocator(cc_ctx *ctx, void *(*alloc)(size_t, void *),
                     void (*free_fn)(void *, void *), void *user);

/*
 * cc_init: create a context from orbital energies and Cholesky vectors.
 *   n_occ, n_virt >= 1; n_aux >= 1.
 *   eps  host double[n]: orbital energies, occupied first. The Fock operator
 *        is taken diagonal, f = diag(eps) (semicanonical spinors, Eqs. 26-27).
 *   L    host complex128 [n_aux][n][n]: Cholesky vectors in the spinor basis
 *        (Eq. 22), each L^P Hermitian in (p, q). The integrals are
 *        <pq||rs> = sum_P (L^P_pr L^P_qs - L^P_ps L^P_qr) (Eq. 23).
 *   out  receives the new context.
 * Errors: CC_ERR_ARG (sizes, NULL pointers), CC_ERR_INPUT (NaN/Inf in eps or
 * L, or L^P not Hermitian to 1e-12 relative), CC_ERR_OOM, CC_ERR_CUDA.
 * The stored integrals with at most two virtual indices (the implementation
 * section's storage policy) are built at the first solver call, in the
 * precision tier current at that point.
 */
int cc_init(int n_occ, int n_virt, int n_aux, const double *eps,
            const double *L, cc_ctx **out);

/* Chunked variant for inputs too large for one host array: create the
 * context with eps, then pass L^P for P in [p0, p1) in any order with
 * cc_add_cholesky (host complex128 [p1-p0][n][n]); the integrals are built at
 * the first solver call once every P has been given (else CC_ERR_STATE). */
int cc_init_chunked(int n_occ, int n_virt, int n_aux, const double *eps,
                    cc_ctx **out);
int cc_add_cholesky(cc_ctx *ctx, int p0, int p1, const double *L_chunk);
/* Same from device memory (L_chunk_dev: complex128 [p1-p0][n][n] on the
 * context's device, complete in the order of the context's stream); the
 * call returns once the chunk has been consumed, so the caller may reuse the
 * buffer. For inputs generated or already resident on the GPU. */
int cc_add_cholesky_dev(cc_ctx *ctx, int p0, int p1, const double *L_chunk_dev);

/* Tier of the CCSD contractions and of the H-bar build (CC_TIER_*; default
 * FP64). Set after ccsd_solve, it also replaces the tier that ccsd_solve
 * finished in for the next H-bar build. */
int cc_set_precision(cc_ctx *ctx, int tier);
/* Tier of the IP-EOM sigma contractions (-1: same as cc_set_precision).
 * The one-body parts of sigma always run in FP64. */
int cc_set_precision_eom(cc_ctx *ctx, int tier);
int cc_set_stream(cc_ctx *ctx, void *stream); /* cudaStream_t */
/* Upper bound (bytes) of the ladder's staging slab of (ac|bd) values formed
 * from L for a block of a (default 4 GiB); the full v^4 tensor is never
 * stored. Smaller budgets mean more, smaller blocks. */
int cc_set_slab_budget(cc_ctx *ctx, size_t bytes);

/* Sizes of the current (possibly truncated) spaces. */
int cc_get_sizes(const cc_ctx *ctx, int *n_occ, int *n_virt, int *n_aux);

/*
 * fns_truncate: frozen natural spinors (Eqs. 24-28).
 * Builds the MP2 virtual-virtual density D_ab (Eq. 24), diagonalises it
 * (Eq. 25), keeps natural spinors with occupation >= threshold, builds and
 * diagonalises F^NS (Eqs. 26-27), forms U = V~ Z~ (Eq. 28, read as
 * V~ times Z~) and rotates the virtual indices of L; eps_virt becomes eps~.
 * threshold >= 0. n_virt_kept (host, may be NULL) receives the new n_virt.
 * Must precede ccsd_solve. Errors: CC_ERR_ARG, CC_ERR_STATE (after CCSD or
 * if nothing would be kept).
 */
int fns_truncate(cc_ctx *ctx, double threshold, int *n_virt_kept);
/* Same, keeping the n_keep natural spinors of largest occupation. */
int fns_truncate_count(cc_ctx *ctx, int n_keep);
/*
 * Streamed natural spinors for systems whose virtual Cholesky block L_vv
 * (X v^2 complex values) does not fit on the device. Call
 * cc_begin_fns_stream right after cc_init_chunked; then
 *   1. pass every P once with cc_add_cholesky: only the L_oo, L_ov and L_vo
 *      blocks are kept (the input is still checked for NaN and Hermiticity);
 *   2. fns_stream_truncate(threshold, n_keep): the Eq. 24 density from MP2
 *      amplitudes formed for one occupied index at a time (the o^2 v^2
 *      amplitudes and <ab||ij> are never held whole), then Eqs. 25-28 as in
 *      fns_truncate; n_keep > 0 keeps that many natural spinors, else those
 *      with occupation >= threshold; n_virt_kept (may be NULL) receives the
 *      count;
 *   3. pass every P once more with cc_add_cholesky: each chunk's L_vv^P is
 *      rotated into the kept basis (U^H L^P U) as it arrives; after the last
 *      one the context continues as after fns_truncate.
 * Solver calls before the second pass ends fail with CC_ERR_STATE.
 */
int cc_begin_fns_stream(cc_ctx *ctx);
int fns_stream_truncate(cc_ctx *ctx, double threshold, int n_keep, int *n_virt_kept);
/* Host double[n_virt_before]: occupations of the last FNS step, descending. */
int fns_get_occupations(const cc_ctx *ctx, double *occ_host, int n);

/*
 * ccsd_solve: CCSD amplitudes (Eqs. 13-14) and energy (Eq. 15).
 * Start t1 = 0, t2 = MP2 (or amplitudes given by cc_set_amplitudes).
 * Jacobi updates with FP64 denominators and Pulay DIIS (8 vectors, from
 * iteration 2). Converged when ||dt||_2 over unique amplitudes < tol and
 * |dE| < tol. In the one-product tiers (TF32, FP16) the residual's rounding
 * leaves a floor under ||dt|| that rises with the amplitudes' size: when the
 * best ||dt|| has not halved for three iterations, the remaining iterations
 * run in the tier's split form (TF32X3, FP16X3), the DIIS history restarts,
 * and cc_get_stats [15] records the iteration.
 * e_corr  host double[2]: complex correlation energy (re, im).
 * n_iter  host int (may be NULL): iterations taken.
 * Errors: CC_ERR_NOT_CONVERGED (results still written), CC_ERR_NUMERIC.
 */
int ccsd_solve(cc_ctx *ctx, double tol, int max_iter, double *e_corr,
               int *n_iter);

/*
 * ipeom_solve: the n_roots IP-EOM-CCSD roots of smallest real part
 * (Eqs. 17-18) by block Davidson with all roots' sigma vectors built in
 * one batch. H-bar elements with at most two virtual indices are built
 * once from the converged amplitudes, in the tier the CCSD iterations
 * finished in (cc_set_precision, or its split form after the move above);
 * the sigma contractions run in the EOM tier (cc_set_precision_eom).
 * omega      host double[n_roots][2]: complex IPs, sorted by real part.
 * r1_weight  host double[n_roots] (may be NULL): ||r1||^2 / ||r||^2.
 * n_iter     host int (may be NULL): Davidson iterations.
 * Converged when every residual ||sigma - omega r||_2 (||r|| = 1) < tol.
 * Errors: CC_ERR_STATE (no converged CCSD), CC_ERR_NOT_CONVERGED.
 */
int ipeom_solve(cc_ctx *ctx, int n_roots, double tol, int max_iter,
                double *omega, double *r1_weight, int *n_iter);

/*
 * ipeom_solve_lr: ipeom_solve's right vectors together with the left ones
 * of Eqs. 19-20. The left vectors solve l^T H-bar = omega l^T with the same
 * block Davidson on the transposed sigma (ipeom_left_sigma_dev), and are
 * then scaled and combined so that the pairs are biorthonormal over the
 * n_roots roots, sum_i l_k^i r_l,i + sum_{i<j,b} l_k^ij_b r_l,ij^b = delta_kl
 * (Eq. 19; bilinear, no complex conjugation). Right vectors have unit
 * 2-norm.
 * omega   host double[n_roots][2]: IPs, sorted by real part.
 * r_host, l_host  host complex128 [n_roots][dim] (may be NULL), the layout
 *   of ipeom_sigma_dev.
 * pole    host double[n_roots][2] (may be NULL): sum_i l^i r_i, the 1h part
 *   of each pair's unit overlap.
 * n_iter  host int[2] (may be NULL): right and left Davidson iterations.
 * Errors: CC_ERR_STATE (no converged CCSD), CC_ERR_NOT_CONVERGED (either
 * Davidson; results written), CC_ERR_NUMERIC (left and right sets do not
 * pair up).
 */
int ipeom_solve_lr(cc_ctx *ctx, int n_roots, double tol, int max_iter,
                   double *omega, double *r_host, double *l_host, double *pole,
                   int *n_iter);

/*
 * cc_batch_ipeom: ipeom_solve for several independent systems (uneven sizes
 * allowed; each context at most once). Their block Davidson iterations run
 * in lockstep; each round builds the sigma vectors of every still-active
 * system in one batched pass whose two-body contractions share one grouped
 * persistent tensor-core launch, replayed from a CUDA graph after its first
 * use (cc_set_graphs). Work runs on systems[0]'s stream.
 * omega [n_sys][n_roots][2], r1_weight [n_sys][n_roots] (may be NULL),
 * n_iter [n_sys] (may be NULL), status [n_sys]: per system CC_OK,
 * CC_ERR_NOT_CONVERGED (iteration limit), or the error that stopped that
 * system alone -- CC_ERR_STATE (no converged CCSD), CC_ERR_ARG (n_roots
 * larger than its IP space), CC_ERR_NUMERIC (its Davidson residual became
 * non-finite); its message is then in cc_last_error(systems[q]) and its
 * omega entries are 0 (or the last Ritz values). The other systems are
 * unaffected: their results equal those of a batch without the failed one.
 * Returns CC_OK, CC_ERR_NOT_CONVERGED if any status is not CC_OK, or an
 * error of the whole call (CC_ERR_CUDA, CC_ERR_OOM, CC_ERR_TIMEOUT; message
 * on systems[0]).
 */
int cc_batch_ipeom(cc_ctx **systems, int n_sys, int n_roots, double tol,
                   int max_iter, double *omega, double *r1_weight, int *n_iter,
                   int *status);
/*
 * cc_batch_solve: CCSD (Eqs. 13-15) then IP-EOM-CCSD (Eqs. 17-18) for
 * several independent systems of uneven size, each context at most once.
 * CCSD runs system after system in each context's own tier (each residual's
 * products already fill the GPU at the sizes batched here); the IP-EOM
 * step is cc_batch_ipeom over the systems whose CCSD converged.
 * e_corr [n_sys][2], omega [n_sys][n_roots][2], r1_weight [n_sys][n_roots]
 * (may be NULL), status [n_sys]: CC_OK, or the first error of that system
 * (its CCSD's CC_ERR_NOT_CONVERGED / CC_ERR_NUMERIC / ..., or its IP-EOM
 * status as in cc_batch_ipeom); a failed system never changes the others'
 * results. Returns CC_OK, CC_ERR_NOT_CONVERGED if any status is not CC_OK,
 * or an error of the whole batched IP-EOM call.
 */
int cc_batch_solve(cc_ctx **systems, int n_sys, int n_roots, double ccsd_tol,
                   double eom_tol, int max_iter, double *e_corr, double *omega,
                   double *r1_weight, int *status);
/* Replay the batched sigma from CUDA graphs (1, default) or not (0). */
int cc_set_graphs(cc_ctx *ctx, int on);

/* Cap on the device bytes the context holds through its allocator (its
 * tensors, workspaces and caches; 0, the default, removes the cap). An
 * allocation beyond the cap fails with CC_ERR_OOM, as does one the device
 * cannot serve. Within the room left (under the cap, and on the device less
 * 2 GiB), ccsd_solve keeps the residual's transient buffers allocatable first
 * and only then holds its optional buffers: the DIIS history (up to 8 pairs,
 * fewer when short of room, none at all when not even one fits), the cache of
 * packed stable operands (otherwise packed again on each use) and a permuted
 * copy of <mb||ej>. The results do not depend on these choices beyond the
 * convergence tolerance. Must not lower the cap below the bytes already held
 * (CC_ERR_ARG). */
int cc_set_memory_limit(cc_ctx *ctx, size_t bytes);

/* Amplitudes as unique elements, host complex128: t1 [o][v] then t2 for
 * i<j, a<b in row-major pair order ([o(o-1)/2][v(v-1)/2]). */
int cc_get_amplitudes(const cc_ctx *ctx, double *t1_host, double *t2_host);
/* Forget amplitudes and H-bar: the next ccsd_solve starts from t1 = 0,
 * t2 = MP2 again (integrals and any FNS truncation are kept). */
int cc_reset_amplitudes(cc_ctx *ctx);
int cc_set_amplitudes(cc_ctx *ctx, const double *t1_host,
                      const double *t2_host);

/*
 * Component entry points (device pointers, context stream, current tier).
 * cc_ladder_dev: out[i][j][a][b] = 1/2 sum_cd <ab||cd> tau[i][j][c][d],
 *   the particle-particle ladder of the doubles equation with <ab||cd> from
 *   the context's virtual Cholesky block (Eq. 23), never stored whole.
 *   tau and out: complex128 [o][o][v][v], tau antisymmetric in (i,j), (c,d).
 *   out is overwritten.
 * cc_residual_dev: one evaluation of the CCSD equations at (t1, t2):
 *   r1 [o][v], r2 [o][o][v][v] (complex128) receive the right-hand sides R
 *   with the Jacobi form t = R / D (D = eps_occ sums minus eps_virt sums).
 * ipeom_sigma_dev: sigma vectors for n_vec packed IP vectors
 *   r[n_vec][dim] -> s[n_vec][dim], dim = o + o(o-1)/2 v, layout r_i then
 *   r_ij^b for i<j (row-major pairs), b fastest. Needs H-bar (ccsd_solve).
 * ipeom_left_sigma_dev: l^T H-bar_IP for n_vec packed left vectors (Eq. 20,
 *   same layout): the transpose of ipeom_sigma_dev's map under the bilinear
 *   pairing of Eq. 19.
 */
int cc_ladder_dev(cc_ctx *ctx, const double *tau_dev, double *out_dev);
int cc_residual_dev(cc_ctx *ctx, const double *t1_dev, const double *t2_dev,
                    double *r1_dev, double *r2_dev);
int ipeom_sigma_dev(cc_ctx *ctx, int n_vec, const double *r_dev,
                    double *s_dev);
int ipeom_left_sigma_dev(cc_ctx *ctx, int n_vec, const double *l_dev,
                         double *s_dev);

/*
 * cc_zgemm_dev: the library's complex GEMM on device buffers,
 *   C[m][n] = sum_k A[m][k] * B[n][k]   (complex128, row-major, C overwritten)
 * in the given tier (CC_TIER_*), on the default stream. The dense
 * contraction core of every step above; exposed for tests and profiling.
 * Allocates its operand planes with cudaMalloc. Errors: CC_ERR_ARG.
 */
int cc_zgemm_dev(int tier, long M, long N, long K, const double *A_dev,
                 const double *B_dev, double *C_dev);

/*
 * cc_cholesky_dev: single-step pivoted Cholesky decomposition (Eq. 21) of
 * the Hermitian positive semidefinite matrix M = B B^H (N x N), which stands
 * for the two-electron integral matrix over orbital pairs; its generator B
 * (device complex128 [N][r], row-major) supplies columns on demand,
 * column p = B conj(B[p]). Step k takes the largest remaining diagonal
 * element d_p and stops when d_p < tau (or after max_vec vectors); otherwise
 * l_k = (M[:,p] - sum_{j<k} l_j conj(l_j[p])) / sqrt(d_p) and d -= |l_k|^2.
 * Every element of M - sum_k l_k l_k^H is then below tau in magnitude.
 * L_dev        device complex128 [max_vec][N]: rows 0..n_vec-1 receive l_k.
 * pivots_host  host long[max_vec] (may be NULL): the pivots p in order.
 * n_vec        host int: vectors formed.
 * FP64 throughout, on the default stream, O(N max_vec) device scratch from
 * the default allocator. Errors: CC_ERR_ARG, CC_ERR_NUMERIC (non-finite
 * diagonal).
 */
int cc_cholesky_dev(long N, int r, const double *B_dev, double tau,
                    int max_vec, double *L_dev, long *pivots_host, int *n_vec);

/*
 * cc_zgemm_noalloc: the same complex GEMM as cc_zgemm_dev, for callers that
 * cannot let the library allocate device memory: host frameworks that
 * reserve nearly all device memory for their own pool (an outside cudaMalloc
 * fails there, or takes memory the framework has promised elsewhere),
 * applications whose device-memory budget is fixed and audited at start-up,
 * and latency-critical loops where cudaMalloc / cudaFree would synchronise
 * the device. (The paper has no counterpart; this is a property of the
 * library interface.)
 *   C[m][n] = sum_k A[m][k] * B[n][k]   (complex128, row-major, C overwritten)
 * A_dev, B_dev, C_dev are device buffers owned by the caller.
 * Temporaries live in one fixed 64 MiB array in device global memory that
 * every GPU loading the library holds until exit; nothing is allocated, no
 * allocating library routine is called, and the tile autotuner
 * (CDFNS_AUTOTUNE) is never run for these calls (cached choices only). The
 * tensor-core tiers need
 * 256 + s (round256(2 M Kp e) + round256(N Kp e)) bytes of it, with
 * Kp = 2K rounded up to 32 (tf32) or 64 (bf16) elements, e = 4 (tf32) or
 * 2 (bf16) bytes and s = 1 (CC_TIER_TF32) or 2 (split tiers); larger
 * problems, and sizes whose byte counts overflow, are rejected with
 * CC_ERR_ARG and a message. CC_TIER_FP16 and CC_TIER_FP16X3 (whose operand
 * scales need device scratch of their own) are rejected with CC_ERR_ARG.
 * CC_TIER_FP64 uses no temporaries. Work runs on the default stream
 * (cc_set_default_stream) and the call returns after it completes.
 * The first call on each device looks up the array's device address with
 * that device current; make that first call before any stream capture.
 * All calls share the array and it keeps the last call's contents: calls
 * whose work could overlap on the GPU (for example from two streams or
 * threads) race on it and must be ordered by the caller.
 * Errors: CC_ERR_ARG, CC_ERR_TIMEOUT, CC_ERR_CUDA (message via
 * cc_last_error(NULL)).
 */
int cc_zgemm_noalloc(int tier, long M, long N, long K, const double *A_dev,
                     const double *B_dev, double *C_dev);

/*
 * cc_selftest_conversions: checks, on the device, the library's integer-pipe
 * FP64 -> FP32 narrowing (IEEE 754 round-to-nearest-even) and FP32 -> FP64
 * widening against the hardware conversion instructions, for every value of
 * x_dev[0..n) (device doubles, not modified). mismatches[0] receives the
 * count of narrowing mismatches, mismatches[1] that of widening mismatches
 * (host array of 2). NaN results compare as equal when both are NaN.
 * Runs on the default stream and returns after it completes.
 * Errors: CC_ERR_ARG (null pointer, n < 0), CC_ERR_CUDA.
 */
int cc_selftest_conversions(const double *x_dev, long n, long long *mismatches);

/*
 * cc_dump_integrals: bit-reproducible FP64 evaluation of Eq. 23 for one
 * block (0: <ij||kl>, 1: <ij||ka>, 2: <ij||ab>, 3: <ia||bj>), host
 * complex128 output in row-major block order. The sum over P runs in
 * ascending order with each complex product formed as
 * (ar*br - ai*bi, ar*bi + ai*br), round-to-nearest, no fused multiply-add,
 * and each term added as (direct - exchange): the result is identical bit
 * for bit to any other evaluation in that order.
 */
int cc_dump_integrals(cc_ctx *ctx, int block, double *out_host);

/* Timing and counters of the last solver calls (host double[n], n <= 24):
 * [0] ladder ms (sum over calls), [1] ladder calls, [2] ladder algorithmic
 * flops per call, [3] fns ms, [4] ccsd ms, [5] ipeom ms, [6] kernel launches
 * since the context was created, [7] ccsd iterations, [8] Davidson
 * iterations, [9] tensor-core GEMM ms inside the ladder, [10] tc GEMM
 * launches inside the ladder, [11] high-water mark of the device bytes the
 * context has held (its own buffers and caches, through its allocator),
 * [12] DIIS pairs held in the last ccsd_solve (8 unless device memory was
 * short), [13] high-water mark of the device bytes held during the CCSD
 * iterations of the last ccsd_solve, [14] device bytes held now, [15] the
 * CCSD iteration after which the residual moved from a one-product tier to
 * its split form (0: it did not), [16] device ms of the IP sigma builds (sum;
 * a batched build is charged to every system in it), [17] sigma builds,
 * [18] algorithmic flops of this system's sigma contractions (8 per complex
 * multiply-add, sum), [19] sigma vectors built, [20..23] reserved (0). */
int cc_get_stats(const cc_ctx *ctx, double *out_host, int n);

/*
 * Learned warm start of the CCSD amplitudes (an extension: the paper has no learned component).
 * A per-element MLP maps gauge-invariant features of each unique doubles
 * element (i<j, a<b) -- log10|t_MP2|, D_ij^ab, <ij||ij>, <ab||ab>, sum and
 * spread of <ia||ia>+<jb||jb> and <ib||ib>+<ja||ja>, eps_i+eps_j, |<ij||ab>|,
 * integrals scaled by the system's rms <ij||ij> and energies by its mean
 * |eps| -- to rho = t_CCSD / t_MP2. Network 8 -> 64 -> 64 -> 2 (ReLU) with
 * FP16 weights and FP32 accumulation; parameters are W1[64][8], b1[64],
 * W2[64][64], b2[64], W3[2][64], b3[2] in that order (host float arrays).
 * The network outputs rho - 1. Training minimises the mean of
 * w |rho_pred - rho|^2 with w = |t_MP2|^2 normalised to mean 1 (the amplitude
 * error), by Adam (beta 0.9/0.999, eps 1e-8) on the GPU.
 */
typedef struct cc_mlp cc_mlp;
int cc_mlp_num_params(void);
int cc_mlp_create(cc_mlp **out);
void cc_mlp_free(cc_mlp *mlp);
const char *cc_mlp_last_error(const cc_mlp *mlp);
int cc_mlp_set_params(cc_mlp *mlp, const float *params_host, int n);
int cc_mlp_get_params(const cc_mlp *mlp, float *params_host, int n);
/* Append up to max_samples evenly strided unique elements of a context with
 * converged CCSD amplitudes to the training set (features and targets). */
int cc_mlp_add_samples(cc_mlp *mlp, cc_ctx *ctx, long max_samples);
int cc_mlp_num_samples(const cc_mlp *mlp, long *n);
/* steps Adam steps on contiguous minibatches of the training set in the
 * order perm_host (perm_len indices, NULL = stored order), wrapping around;
 * final_loss (may be NULL) gets the last minibatch loss. */
int cc_mlp_train(cc_mlp *mlp, int steps, int batch, float lr,
                 const int *perm_host, long perm_len, double *final_loss);
/* Loss and gradient for a given batch: X_host [n][8], Y_host [n][3] holding
 * (Re, Im of the target rho - 1, weight); grad_host [num_params]. */
int cc_mlp_loss_grad(cc_mlp *mlp, long n, const float *X_host,
                     const float *Y_host, double *loss, float *grad_host);
/* Features of the first n unique elements of a context (host [n][8]). */
int cc_mlp_features(cc_ctx *ctx, long n, float *X_host);
/* Set the context's starting amplitudes t1 = 0, t2 = rho(MLP) * t_MP2; the
 * next ccsd_solve starts from them. Errors: CC_ERR_STATE after ccsd_solve. */
int cc_mlp_warm_start(cc_mlp *mlp, cc_ctx *ctx);

/*
 * Test hooks for the error paths (no counterpart in the paper).
 * cc_set_wait_limit: limit (ns) of every pipeline wait inside the
 *   tensor-core kernels launched from now on, process-wide; 0 restores the
 *   default of 2 s. A wait that runs out makes the kernel record an error
 *   flag, wait (2 s at most) for its own copies and MMAs in flight, free its
 *   tensor memory and return; the call then fails with CC_ERR_TIMEOUT and the
 *   context stays usable. A limit of a few ns makes the first wait that does
 *   not succeed at once run out.
 * cc_set_fault_injection: kind 1 writes a NaN into the CCSD residual of
 *   iteration at_iteration (ccsd_solve then fails with CC_ERR_NUMERIC); kind
 *   2 writes one into the sigma vectors of Davidson iteration at_iteration
 *   (ipeom_solve fails with CC_ERR_NUMERIC; in cc_batch_ipeom only this
 *   system stops); 0 switches injection off. Host-side: the value is copied
 *   into device memory between kernels. Fires once.
 */
int cc_set_wait_limit(unsigned long long ns);
int cc_set_fault_injection(cc_ctx *ctx, int kind, int at_iteration);

/*
 * Davidson starting vectors (an extension beyond the paper, which names the
 * Davidson method without a start). The n_roots lowest diagonal elements of
 * H-bar_IP seed the roots. Mode 0 (default): unit vectors there. Mode 1: a
 * root seeded at a 1h element i starts from r_i = 1 plus the first-order
 * (Rayleigh-Schroedinger) 2h1p components c_nu = M_nu,i / (d_i - d_nu)
 * about the diagonal d (M_nu,i = -W_ibjk for nu = (j<k, b)); roots seeded at
 * 2h1p elements keep unit vectors. Mode 2: the components are rho_nu c_nu
 * with rho_nu from a trained network (cc_mlp, same architecture as the
 * amplitude warm start, features listed at cc_mlp_guess_features). The
 * roots do not depend on the start; it changes the iteration count only.
 * The network must outlive its use by the context.
 */
int cc_set_davidson_guess(cc_ctx *ctx, int mode, const cc_mlp *mlp);
/* The n_roots starting vectors of the current mode before orthonormalisation
 * (device complex128 [n_roots][dim], the ipeom_sigma_dev layout). Needs a
 * converged ccsd_solve; builds H-bar if needed. */
int ipeom_guess_dev(cc_ctx *ctx, int n_roots, double *out_dev);
/* Features of the first n 2h1p elements (j<k row-major, b fastest) for a
 * root seeded at 1h element `seed` (host float [n][8]): log10|c_nu|,
 * Re(d_i - d_nu) / d_scale, |W_ibjk| / g_scale, [seed is j or k],
 * Re(d_i) / d_scale, <jk||jk> / g_scale, (<jb||jb> + <kb||kb>) / g_scale,
 * |<jb||jb> - <kb||kb>| / g_scale, with the scales of the amplitude
 * features. */
int cc_mlp_guess_features(cc_ctx *ctx, int seed, long n, float *X_host);
/* Training samples for the learned start from the right vectors of the
 * context's last converged ipeom_solve: for every root whose 1h weight is at
 * least one half, seeded at its largest 1h element i and scaled to r_i = 1,
 * the targets rho_nu = r_nu / c_nu (up to max_samples evenly strided
 * elements; weights |c_nu|^2 normalised to mean one). */
int cc_mlp_add_guess_samples(cc_mlp *mlp, cc_ctx *ctx, long max_samples);

const char *cc_last_error(const cc_ctx *ctx); /* NULL ctx: last global */
void cc_free(cc_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* CDFNS_H */
