// Single-step pivoted Cholesky decomposition (Eq. 21) on the GPU.
//
// The matrix is Hermitian positive semidefinite, M = B B^H (N x N), given by
// a generator B [N][r] whose columns stand in for two-electron integrals
// computed on demand: column p of M is B conj(B[p]). Step k picks the largest
// remaining diagonal element d_p, stops when d_p < tau, and otherwise forms
//   l_k = (M[:, p] - sum_{j<k} l_j conj(l_j[p])) / sqrt(d_p),  d -= |l_k|^2.
// Every element of M - sum_k l_k l_k^H is then below tau in magnitude (the
// remainder is positive semidefinite with every diagonal element below tau).
//
// The vectors are accumulated pair-major, Lt[q][k] (row stride ld), so that
// both products of a step are row-contiguous matrix-vector products: the
// column of M over B's rows, and the correction over the k vectors so far.
// Both run on the contraction engine's FP64 GEMV kernels; the argmax is a
// two-pass block reduction whose partial results the host finishes (one
// short copy per step). The decomposition is bound by HBM bandwidth: each
// step reads B and the vectors formed so far once.
#include <algorithm>
#include <cmath>
#include <vector>

#include "engine.h"

namespace cdfns {

namespace {

constexpr int ARGMAX_THREADS = 256;
constexpr int ARGMAX_BLOCKS = 1024;

// d[q] = sum_s |B[q][s]|^2
__global__ void row_norm2_kernel(const double2 *__restrict__ B, long N, int r, double *d) {
  for (long q = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; q < N;
       q += static_cast<long>(gridDim.x) * blockDim.x) {
    const double2 *row = B + q * r;
    double s = 0.0;
    for (int j = 0; j < r; ++j) s += row[j].x * row[j].x + row[j].y * row[j].y;
    d[q] = s;
  }
}

// per block: the largest d and its smallest index
__global__ void __launch_bounds__(ARGMAX_THREADS)
    block_argmax_kernel(const double *__restrict__ d, long N, double *bv, long *bi) {
  __shared__ double sv[ARGMAX_THREADS];
  __shared__ long si[ARGMAX_THREADS];
  double v = -1.0;
  long idx = -1;
  for (long q = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; q < N;
       q += static_cast<long>(gridDim.x) * blockDim.x) {
    if (d[q] > v) {  // ascending q per thread: the first of equal values stays
      v = d[q];
      idx = q;
    }
  }
  sv[threadIdx.x] = v;
  si[threadIdx.x] = idx;
  __syncthreads();
  for (int h = ARGMAX_THREADS / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      const double v2 = sv[threadIdx.x + h];
      const long i2 = si[threadIdx.x + h];
      if (v2 > sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 >= 0 && i2 < si[threadIdx.x])) {
        sv[threadIdx.x] = v2;
        si[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    bv[blockIdx.x] = sv[0];
    bi[blockIdx.x] = si[0];
  }
}

// l = s * col; Lt[q][k] = l; d[q] -= |l|^2
__global__ void store_vector_kernel(const double2 *__restrict__ col, double s, long N, double2 *Lt,
                                    long ld, int k, double *d) {
  for (long q = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; q < N;
       q += static_cast<long>(gridDim.x) * blockDim.x) {
    const double2 l = make_double2(s * col[q].x, s * col[q].y);
    Lt[q * ld + k] = l;
    d[q] -= l.x * l.x + l.y * l.y;
  }
}

unsigned blocks_for(long n) {
  return static_cast<unsigned>(std::max<long>(1, std::min<long>((n + 255) / 256, 4096)));
}

}  // namespace

int pivoted_cholesky(const cplx *B, long N, int r, double tau, int max_vec, cplx *L, long *piv,
                     Allocator *al, cudaStream_t st, int num_sms) {
  Engine eng;
  eng.al = al;
  eng.st = st;
  eng.num_sms = num_sms;
  const long ld = max_vec;
  Buf d(al, sizeof(double) * N), col(al, sizeof(cplx) * N), Lt(al, sizeof(cplx) * N * ld);
  const unsigned nb = static_cast<unsigned>(std::min<long>(ARGMAX_BLOCKS, (N + 255) / 256));
  Buf bv(al, sizeof(double) * nb), bi(al, sizeof(long) * nb);
  std::vector<double> hv(nb);
  std::vector<long> hi(nb);
  row_norm2_kernel<<<blocks_for(N), 256, 0, st>>>(reinterpret_cast<const double2 *>(B), N, r,
                                                  d.as<double>());
  LAUNCH_CHECK();
  count_launch();
  int k = 0;
  for (; k < max_vec; ++k) {
    block_argmax_kernel<<<nb, ARGMAX_THREADS, 0, st>>>(d.as<double>(), N, bv.as<double>(),
                                                       bi.as<long>());
    LAUNCH_CHECK();
    count_launch();
    CUDA_CHECK(cudaMemcpyAsync(hv.data(), bv.p, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaMemcpyAsync(hi.data(), bi.p, sizeof(long) * nb, cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaStreamSynchronize(st));
    double dmax = -1.0;
    long p = -1;
    for (unsigned b = 0; b < nb; ++b)
      if (hi[b] >= 0 && (hv[b] > dmax || (hv[b] == dmax && hi[b] < p))) {
        dmax = hv[b];
        p = hi[b];
      }
    if (p >= 0 && !std::isfinite(dmax)) fail(CC_ERR_NUMERIC, "cholesky: non-finite diagonal");
    if (p < 0 || !(dmax >= tau) || !(dmax > 0.0)) break;
    // column p of M = B conj(B[p])
    eng.contract(C1(), T(B, "qs", {N, r}), conj(T(B + p * r, "s", {r})), C0(), T(col.c(), "q", {N}),
                 TIER_FP64);
    // minus sum_{j<k} l_j conj(l_j[p])
    if (k > 0)
      eng.contract(Cr(-1), Tv(Lt.c(), "qj", {N, k}, {ld, 1}), conj(Tv(Lt.c() + p * ld, "j", {k}, {1})),
                   C1(), T(col.c(), "q", {N}), TIER_FP64);
    store_vector_kernel<<<blocks_for(N), 256, 0, st>>>(reinterpret_cast<const double2 *>(col.p),
                                                       1.0 / std::sqrt(dmax), N, Lt.as<double2>(),
                                                       ld, k, d.as<double>());
    LAUNCH_CHECK();
    count_launch();
    if (piv) piv[k] = p;
  }
  // vectors row-major for the caller: L[k][q]
  if (k > 0)
    eng.permute_into(C1(), Tv(Lt.c(), "qk", {N, k}, {ld, 1}), C0(), T(L, "kq", {k, N}));
  CUDA_CHECK(cudaStreamSynchronize(st));
  return k;
}

}  // namespace cdfns
