// Generic tensor helpers: offset tables, scaling, permutations, reductions.
#include <algorithm>

#include "kernels.h"

#include <type_traits>

namespace cdfns {

std::atomic<unsigned long long> g_launches{0};
thread_local unsigned long long t_launches = 0;

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

// y = a x + b y. Real coefficients take two FP64 operations per component
// instead of a complex multiply (GB300's FP64 pipe, not memory, otherwise
// bounds this kernel); a = +-1 with b = 1 only adds.
template <int MODE>  // 0 complex a, b; 1 real a, b; 2 y +- x (sign in a.x)
__global__ void axpby_kernel(long n, double2 a, const double2 *x, double2 b, double2 *y) {
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    const double2 xv = x[i];
    if (MODE == 2) {
      const double2 yv = y[i];
      y[i] = a.x > 0 ? make_double2(yv.x + xv.x, yv.y + xv.y) : make_double2(yv.x - xv.x, yv.y - xv.y);
    } else if (MODE == 1) {
      if (b.x == 0.0) {
        y[i] = make_double2(a.x * xv.x, a.x * xv.y);
      } else {
        const double2 yv = y[i];
        y[i] = make_double2(fma(a.x, xv.x, b.x * yv.x), fma(a.x, xv.y, b.x * yv.y));
      }
    } else {
      const double2 yy = (b.x == 0.0 && b.y == 0.0) ? make_double2(0.0, 0.0) : cmul(b, y[i]);
      y[i] = cadd(cmul(a, xv), yy);
    }
  }
}

// I: the index type of the digit arithmetic (32-bit when every index fits:
// 64-bit division is a long instruction sequence). Four elements per thread
// and pass, their loads issued before the stores (in and out never overlap).
template <typename I>
__global__ void permute_kernel(double2 *__restrict__ out, const double2 *__restrict__ in,
                               long total, Dims D, double2 alpha, double2 beta, bool conj) {
  const long stride = static_cast<long>(gridDim.x) * blockDim.x;
  const bool pm1 = alpha.y == 0.0 && (alpha.x == 1.0 || alpha.x == -1.0);
  const bool b1 = beta.x == 1.0 && beta.y == 0.0, b0 = beta.x == 0.0 && beta.y == 0.0;
  for (long i0 = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i0 < total;
       i0 += 4 * stride) {
    double2 x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long i = i0 + u * stride;
      if (i >= total) break;
      long off = 0;
      if (D.nd == 1) {
        off = i * D.s[0];
      } else {
        I rem = static_cast<I>(i);
        for (int k = D.nd - 1; k >= 0; --k) {
          const I dk = static_cast<I>(D.d[k]);
          const I q = rem / dk;
          off += static_cast<long>(rem - q * dk) * D.s[k];
          rem = q;
        }
      }
      x[u] = in[off];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long i = i0 + u * stride;
      if (i >= total) break;
      double2 v = x[u];
      if (conj) v.y = -v.y;
      // +-1 scalings and beta in {0, 1} without FP64 multiplies (GB300's
      // FP64 rate makes them the cost of this memory-bound kernel)
      if (pm1) {
        if (alpha.x < 0) v = make_double2(-v.x, -v.y);
      } else {
        v = cmul(alpha, v);
      }
      if (b1) v = cadd(v, out[i]);
      else if (!b0) v = cadd(v, cmul(beta, out[i]));
      out[i] = v;
    }
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

// m dot products <x_k|y> (k < m <= 16) in one pass over y. F32: products
// and per-thread sums in FP32 (operands narrowed on the integer pipes), block
// sums in FP64; for the tensor-core tiers, whose B matrices only steer DIIS.
struct PtrList {
  const double2 *p[16];
};
template <bool F32>
__global__ void __launch_bounds__(256) dot_multi_partial(PtrList xs, int m, const double2 *y, long n,
                                                         double2 *partial) {
  using A = typename std::conditional<F32, float, double>::type;
  A ar[16], ai[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) ar[k] = ai[k] = A(0);
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    const double2 yv = y[i];
    A yr, yi;
    if (F32) {
      yr = f64_to_f32(yv.x);
      yi = f64_to_f32(yv.y);
    } else {
      yr = yv.x;
      yi = yv.y;
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      if (k < m) {
        const double2 xv = xs.p[k][i];
        A xr, xi;
        if (F32) {
          xr = f64_to_f32(xv.x);
          xi = f64_to_f32(xv.y);
        } else {
          xr = xv.x;
          xi = xv.y;
        }
        // conj(x) y
        ar[k] = fma(xr, yr, fma(xi, yi, ar[k]));
        ai[k] = fma(xr, yi, fma(-xi, yr, ai[k]));
      }
    }
  }
  for (int k = 0; k < m; ++k) {
    double2 v = make_double2(F32 ? f32_to_f64(static_cast<float>(ar[k])) : static_cast<double>(ar[k]),
                             F32 ? f32_to_f64(static_cast<float>(ai[k])) : static_cast<double>(ai[k]));
    v = block_sum(v);
    if (threadIdx.x == 0) partial[static_cast<long>(k) * gridDim.x + blockIdx.x] = v;
    __syncthreads();
  }
}

__global__ void dot_multi_final(const double2 *partial, int np, int m, double2 *res, long stride) {
  for (int k = 0; k < m; ++k) {
    double2 acc = make_double2(0.0, 0.0);
    for (int i = threadIdx.x; i < np; i += blockDim.x) acc = cadd(acc, partial[static_cast<long>(k) * np + i]);
    acc = block_sum(acc);
    if (threadIdx.x == 0) res[k * stride] = acc;
    __syncthreads();
  }
}

__global__ void dot_final(const double2 *partial, int np, double2 *res) {
  double2 acc = make_double2(0.0, 0.0);
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc = cadd(acc, partial[i]);
  acc = block_sum(acc);
  if (threadIdx.x == 0) *res = acc;
}

// R += c * P(X) for P = P(ij) (mode 1), P(ab) (mode 2) or P(ij)P(ab)
// (mode 3), X and R [o][o][v][v]. One block owns every image of its 16 x 16
// (a, b) tile: the pairs (i,j)/(j,i) for modes 1 and 3 and the tiles
// (A,B)/(B,A) for modes 2 and 3. It reads each X element once and reads and
// writes each R element once; transposed tiles go through shared memory so
// all global accesses run along b.
__global__ void antisym_add_kernel(double2 *R, const double2 *X, int o, int v, double c, int mode,
                                   int ntile, bool unit_c) {
  __shared__ double2 sx[4][16][17];
  const int tx = threadIdx.x, ty = threadIdx.y;
  // (i, j): i < j for modes 1 and 3 (i == j adds nothing), all pairs for mode 2
  int i, j;
  if (mode & 1) {
    int p = blockIdx.z;
    i = 0;
    while (p >= o - 1 - i) {
      p -= o - 1 - i;
      ++i;
    }
    j = i + 1 + p;
  } else {
    i = blockIdx.z / o;
    j = blockIdx.z - i * o;
  }
  // (A, B) tiles: A <= B for modes 2 and 3, all tiles for mode 1
  int ta, tb;
  if (mode & 2) {
    int p = blockIdx.x;
    ta = 0;
    while (p >= ntile - ta) {
      p -= ntile - ta;
      ++ta;
    }
    tb = ta + p;
  } else {
    ta = blockIdx.x / ntile;
    tb = blockIdx.x - ta * ntile;
  }
  const long vv = static_cast<long>(v) * v;
  const long bij = (static_cast<long>(i) * o + j) * vv, bji = (static_cast<long>(j) * o + i) * vv;
  const int a0 = ta * 16, b0 = tb * 16;
  // direct tile (row a0 + ty, column b0 + tx) and transposed tile (row b0 + ty, column a0 + tx)
  const int ra = a0 + ty, cb = b0 + tx, rb = b0 + ty, ca = a0 + tx;
  const bool in_d = ra < v && cb < v, in_t = rb < v && ca < v;
  const long ed = static_cast<long>(ra) * v + cb, et = static_cast<long>(rb) * v + ca;
  const double2 z = make_double2(0.0, 0.0);
  // sx[0]: X[ij] direct, sx[1]: X[ji] direct, sx[2]: X[ij] transposed, sx[3]: X[ji] transposed
  const double2 x_ij = in_d ? X[bij + ed] : z;
  const double2 x_ji = (mode & 1) && in_d ? X[bji + ed] : z;
  if (mode & 2) {
    sx[2][ty][tx] = in_t ? X[bij + et] : z;
    if (mode & 1) sx[3][ty][tx] = in_t ? X[bji + et] : z;
  }
  __syncthreads();
  // Y(a, b) for a = ra, b = cb
  double2 y = x_ij;
  if (mode & 1) y = csub(y, x_ji);
  if (mode & 2) {
    y = csub(y, sx[2][tx][ty]);                 // X[ij][b][a]
    if (mode & 1) y = cadd(y, sx[3][tx][ty]);   // X[ji][b][a]
  }
  // c = 1 (the usual case) costs no FP64 multiplications
  if (!unit_c) y = cscale(c, y);
  const bool diag_tile = (mode & 2) && ta == tb;
  // direct images: R[ij][ab] += Y, R[ji][ab] -= Y (mode 1/3)
  // (on a diagonal tile only a < b is handled here; a == b adds nothing)
  if (in_d && !(diag_tile && ra >= cb)) {
    R[bij + ed] = cadd(R[bij + ed], y);
    if (mode & 1) R[bji + ed] = csub(R[bji + ed], y);
  }
  if (!(mode & 2)) return;
  // transposed images: R[ij][ba] -= Y, R[ji][ba] += Y, written along a
  sx[0][ty][tx] = y;
  __syncthreads();
  if (in_t) {
    const double2 yt = sx[0][tx][ty];  // Y(a = ca, b = rb)
    if (!(diag_tile && ca >= rb)) {
      R[bij + et] = csub(R[bij + et], yt);
      if (mode & 1) R[bji + et] = cadd(R[bji + et], yt);
    }
  }
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
  const bool real = alpha.y == 0.0 && beta.y == 0.0;
  if (real && (alpha.x == 1.0 || alpha.x == -1.0) && beta.x == 1.0)
    axpby_kernel<2><<<grid_for(n), 256, 0, st>>>(n, alpha, x, beta, y);
  else if (real)
    axpby_kernel<1><<<grid_for(n), 256, 0, st>>>(n, alpha, x, beta, y);
  else
    axpby_kernel<0><<<grid_for(n), 256, 0, st>>>(n, alpha, x, beta, y);
  LAUNCH_CHECK();
  count_launch();
}

void permute(cplx *out, const cplx *in, int nd, const long *odims, const long *istr, cplx alpha,
             cplx beta, bool conj, cudaStream_t st) {
  if (nd > MAXD) fail(CC_ERR_ARG, "permute: rank too large");
  Dims D;
  D.nd = 0;
  long total = 1;
  // drop unit dims and merge neighbours that are contiguous in the input too
  // (out is row-major): an identity layout becomes one dimension
  for (int i = 0; i < nd; ++i) {
    total *= odims[i];
    if (odims[i] == 1) continue;
    if (D.nd > 0 && D.s[D.nd - 1] == istr[i] * odims[i]) {
      D.d[D.nd - 1] *= odims[i];
      D.s[D.nd - 1] = istr[i];
    } else {
      D.d[D.nd] = odims[i];
      D.s[D.nd] = istr[i];
      ++D.nd;
    }
  }
  if (total <= 0) return;
  if (D.nd == 0) {
    D.nd = 1;
    D.d[0] = 1;
    D.s[0] = 0;
  }
  if (total <= 0xffffffffL)
    permute_kernel<unsigned><<<grid_for(total), 256, 0, st>>>(out, in, total, D, alpha, beta, conj);
  else
    permute_kernel<unsigned long long><<<grid_for(total), 256, 0, st>>>(out, in, total, D, alpha,
                                                                        beta, conj);
  LAUNCH_CHECK();
  count_launch();
}

void antisym_add(cplx *R, const cplx *X, int o, int v, double c, int mode, cudaStream_t st) {
  if (o <= 0 || v <= 0) return;
  if (mode < 1 || mode > 3) fail(CC_ERR_ARG, "antisym_add: bad mode");
  const long pairs = (mode & 1) ? static_cast<long>(o) * (o - 1) / 2 : static_cast<long>(o) * o;
  if (pairs == 0) return;
  if (pairs > 65535) fail(CC_ERR_ARG, "antisym_add: n_occ too large");
  const int nt = (v + 15) / 16;
  const long tiles = (mode & 2) ? static_cast<long>(nt) * (nt + 1) / 2 : static_cast<long>(nt) * nt;
  dim3 grid(static_cast<unsigned>(tiles), 1, static_cast<unsigned>(pairs));
  antisym_add_kernel<<<grid, dim3(16, 16), 0, st>>>(R, X, o, v, c, mode, nt, c == 1.0);
  LAUNCH_CHECK();
  count_launch();
}

void dot_multi(const cplx *const *xs, int m, const cplx *y, long n, bool f32, cplx *res,
               long res_stride, cplx *scratch, long scratch_len, cudaStream_t st) {
  if (m <= 0) return;
  if (m > 16) fail(CC_ERR_ARG, "dot_multi: at most 16 vectors");
  PtrList pl;
  for (int k = 0; k < 16; ++k) pl.p[k] = k < m ? xs[k] : nullptr;
  int nb = static_cast<int>(std::max<long>(1, std::min<long>(RED_BLOCKS, (n + 255) / 256)));
  nb = static_cast<int>(std::min<long>(nb, scratch_len / m));
  if (nb < 1) fail(CC_ERR_ARG, "dot_multi: scratch too small");
  if (f32)
    dot_multi_partial<true><<<nb, RED_THREADS, 0, st>>>(pl, m, y, n, scratch);
  else
    dot_multi_partial<false><<<nb, RED_THREADS, 0, st>>>(pl, m, y, n, scratch);
  LAUNCH_CHECK();
  dot_multi_final<<<1, RED_THREADS, 0, st>>>(scratch, nb, m, res, res_stride);
  LAUNCH_CHECK();
  count_launch(2);
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
