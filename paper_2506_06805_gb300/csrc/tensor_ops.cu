// Generic tensor helpers: offset tables, scaling, permutations, reductions.
#include <algorithm>

#include "kernels.h"

namespace cdfns {

unsigned long long g_launches = 0;

namespace {

constexpr int MAXD = 8;
struct Dims {
  int nd;
  long d[MAXD];
  long s[MAXD];
};

__global__ void offsets_kernel(long *table, long total, Dims D) {
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    long rem = i, off = 0;
    for (int k = D.nd - 1; k >= 0; --k) {
      const long digit = rem % D.d[k];
      rem /= D.d[k];
      off += digit * D.s[k];
    }
    table[i] = off;
  }
}

__global__ void scale2d_kernel(double2 *C, const long *cm, const long *cn, long ldc, long M, long N,
                               double2 beta) {
  const long total = M * N;
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    const long m = i / N, n = i % N;
    const long off = (cm ? cm[m] : m * ldc) + (cn ? cn[n] : n);
    C[off] = (beta.x == 0.0 && beta.y == 0.0) ? make_double2(0.0, 0.0) : cmul(beta, C[off]);
  }
}

__global__ void axpby_kernel(long n, double2 a, const double2 *x, double2 b, double2 *y) {
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    const double2 yy = (b.x == 0.0 && b.y == 0.0) ? make_double2(0.0, 0.0) : cmul(b, y[i]);
    y[i] = cadd(cmul(a, x[i]), yy);
  }
}

__global__ void permute_kernel(double2 *out, const double2 *in, long total, Dims D, double2 alpha,
                               double2 beta, bool conj) {
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    long rem = i, off = 0;
    for (int k = D.nd - 1; k >= 0; --k) {
      const long digit = rem % D.d[k];
      rem /= D.d[k];
      off += digit * D.s[k];
    }
    double2 x = in[off];
    if (conj) x.y = -x.y;
    // +-1 scalings and beta in {0, 1} without FP64 multiplies (GB300's FP64
    // rate makes them the cost of this memory-bound kernel)
    if (alpha.y == 0.0 && (alpha.x == 1.0 || alpha.x == -1.0)) {
      if (alpha.x < 0) x = make_double2(-x.x, -x.y);
    } else {
      x = cmul(alpha, x);
    }
    if (beta.x == 1.0 && beta.y == 0.0) x = cadd(x, out[i]);
    else if (!(beta.x == 0.0 && beta.y == 0.0)) x = cadd(x, cmul(beta, out[i]));
    out[i] = x;
  }
}

// Block-level deterministic reduction of sum conj?(x) y.
constexpr int RED_BLOCKS = 1024;
constexpr int RED_THREADS = 256;

__device__ double2 block_sum(double2 v) {
  __shared__ double2 sh[RED_THREADS / 32];
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = l < RED_THREADS / 32 ? sh[l] : make_double2(0.0, 0.0);
    for (int o = 16; o > 0; o >>= 1) {
      v.x += __shfl_down_sync(0xffffffffu, v.x, o);
      v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
  }
  return v;
}

__global__ void dot_partial(const double2 *x, const double2 *y, long n, bool conj_x,
                            double2 *partial) {
  double2 acc = make_double2(0.0, 0.0);
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    double2 a = x[i];
    if (conj_x) a.y = -a.y;
    acc = cfma(a, y[i], acc);
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void dot_final(const double2 *partial, int np, double2 *res) {
  double2 acc = make_double2(0.0, 0.0);
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc = cadd(acc, partial[i]);
  acc = block_sum(acc);
  if (threadIdx.x == 0) *res = acc;
}

__global__ void antisym_add_kernel(double2 *R, const double2 *X, int o, int v, double c, int mode) {
  __shared__ double2 t1[16][17];
  __shared__ double2 t2[16][17];
  const int i = blockIdx.z / o, j = blockIdx.z % o;
  const int a0 = blockIdx.y * 16, b0 = blockIdx.x * 16;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const long vv = static_cast<long>(v) * v;
  const long ij = (static_cast<long>(i) * o + j) * vv;
  const long ji = (static_cast<long>(j) * o + i) * vv;
  if (mode & 2) {
    // tiles of X[..][b][a] read along a (coalesced) and used transposed
    const int bb = b0 + ty, aa = a0 + tx;
    const bool in = bb < v && aa < v;
    t1[ty][tx] = in ? X[ij + static_cast<long>(bb) * v + aa] : make_double2(0.0, 0.0);
    if (mode & 1) t2[ty][tx] = in ? X[ji + static_cast<long>(bb) * v + aa] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const int a = a0 + ty, b = b0 + tx;
  if (a >= v || b >= v) return;
  const long e = static_cast<long>(a) * v + b;
  double2 x = X[ij + e];
  if (mode & 1) x = csub(x, X[ji + e]);
  if (mode & 2) {
    x = csub(x, t1[tx][ty]);
    if (mode & 1) x = cadd(x, t2[tx][ty]);
  }
  if (c == 1.0) R[ij + e] = cadd(R[ij + e], x);
  else if (c == -1.0) R[ij + e] = csub(R[ij + e], x);
  else R[ij + e] = cadd(R[ij + e], cscale(c, x));
}

inline unsigned grid_for(long n, int threads = 256) {
  return static_cast<unsigned>(std::max<long>(1, std::min<long>((n + threads - 1) / threads, 152L * 64)));
}

}  // namespace

void make_offsets(long *table, int nd, const long *dims, const long *strides, cudaStream_t st) {
  if (nd > MAXD) fail(CC_ERR_ARG, "make_offsets: rank too large");
  Dims D;
  D.nd = nd;
  long total = 1;
  for (int i = 0; i < nd; ++i) {
    D.d[i] = dims[i];
    D.s[i] = strides[i];
    total *= dims[i];
  }
  if (nd == 0) {
    D.nd = 0;
    total = 1;
  }
  offsets_kernel<<<grid_for(total), 256, 0, st>>>(table, total, D);
  LAUNCH_CHECK();
  count_launch();
}

void scale_2d(cplx *C, const long *cm, const long *cn, long ldc, long M, long N, cplx beta,
              cudaStream_t st) {
  if (M <= 0 || N <= 0) return;
  if (beta.x == 1.0 && beta.y == 0.0) return;
  scale2d_kernel<<<grid_for(M * N), 256, 0, st>>>(C, cm, cn, ldc, M, N, beta);
  LAUNCH_CHECK();
  count_launch();
}

void axpby(long n, cplx alpha, const cplx *x, cplx beta, cplx *y, cudaStream_t st) {
  if (n <= 0) return;
  axpby_kernel<<<grid_for(n), 256, 0, st>>>(n, alpha, x, beta, y);
  LAUNCH_CHECK();
  count_launch();
}

void permute(cplx *out, const cplx *in, int nd, const long *odims, const long *istr, cplx alpha,
             cplx beta, bool conj, cudaStream_t st) {
  if (nd > MAXD) fail(CC_ERR_ARG, "permute: rank too large");
  Dims D;
  D.nd = nd;
  long total = 1;
  for (int i = 0; i < nd; ++i) {
    D.d[i] = odims[i];
    D.s[i] = istr[i];
    total *= odims[i];
  }
  if (total <= 0) return;
  permute_kernel<<<grid_for(total), 256, 0, st>>>(out, in, total, D, alpha, beta, conj);
  LAUNCH_CHECK();
  count_launch();
}

void antisym_add(cplx *R, const cplx *X, int o, int v, double c, int mode, cudaStream_t st) {
  if (o <= 0 || v <= 0) return;
  if (static_cast<long>(o) * o > 65535) fail(CC_ERR_ARG, "antisym_add: n_occ too large");
  dim3 grid((v + 15) / 16, (v + 15) / 16, o * o);
  antisym_add_kernel<<<grid, dim3(16, 16), 0, st>>>(R, X, o, v, c, mode);
  LAUNCH_CHECK();
  count_launch();
}

void dot_dev(const cplx *x, const cplx *y, long n, bool conj_x, cplx *res, cudaStream_t st,
             cplx *scratch) {
  const int nb = static_cast<int>(std::max<long>(1, std::min<long>(RED_BLOCKS, (n + 255) / 256)));
  dot_partial<<<nb, RED_THREADS, 0, st>>>(x, y, n, conj_x, scratch);
  LAUNCH_CHECK();
  dot_final<<<1, RED_THREADS, 0, st>>>(scratch, nb, res);
  LAUNCH_CHECK();
  count_launch(2);
}

cplx dot(const cplx *x, const cplx *y, long n, bool conj_x, cudaStream_t st, cplx *scratch,
         cplx *host_out) {
  dot_dev(x, y, n, conj_x, scratch + RED_BLOCKS, st, scratch);
  cplx h;
  CUDA_CHECK(cudaMemcpyAsync(&h, scratch + RED_BLOCKS, sizeof(cplx), cudaMemcpyDeviceToHost, st));
  CUDA_CHECK(cudaStreamSynchronize(st));
  if (host_out) *host_out = h;
  return h;
}

}  // namespace cdfns
