// Complex FP64 GEMM on the FP64 pipe (the plain CC_TIER_FP64 path).
//
// C(m, n) = alpha * sum_k A(m, k) B(n, k) + beta * C(m, n) with operands
// gathered through offset tables (see GemmDesc). 64 x 64 complex output tile
// per 256-thread CTA, 4 x 4 complex accumulators per thread, K staged through
// shared memory 8 complex elements at a time. GB300's FP64 rate is low enough
// that this register tiling keeps the FP64 pipe busy; split-K over
// blockIdx.z (with FP64 atomics) covers tall-skinny shapes such as the
// Davidson subspace products.
#include <algorithm>

#include "kernels.h"

namespace cdfns {
namespace {

constexpr int TM = 64, TN = 64, TK = 8;

__global__ void __launch_bounds__(256)
    zgemm_kernel(long M, long N, long K, const double2 *__restrict__ A, const long *__restrict__ am,
                 const long *__restrict__ ak, long lda, bool conjA, const double2 *__restrict__ B,
                 const long *__restrict__ bn, const long *__restrict__ bk, long ldb, bool conjB,
                 double2 *C, const long *__restrict__ cm, const long *__restrict__ cn, long ldc,
                 double2 alpha, double2 beta, long k_per_split, bool atomic) {
  __shared__ double2 As[TK][TM + 1];
  __shared__ double2 Bs[TK][TN + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const long m0 = static_cast<long>(blockIdx.y) * TM;
  const long n0 = static_cast<long>(blockIdx.x) * TN;
  const long kbeg = static_cast<long>(blockIdx.z) * k_per_split;
  const long kend = min(K, kbeg + k_per_split);

  // loader mapping: 256 threads x 2 elements = 64 rows x 8 k
  const int lr = threadIdx.x >> 2;        // row within tile
  const int lk = (threadIdx.x & 3) * 2;   // k pair
  const long arow = m0 + lr, brow = n0 + lr;
  const long aro = arow < M ? (am ? am[arow] : arow * lda) : -1;
  const long bro = brow < N ? (bn ? bn[brow] : brow * ldb) : -1;

  double2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);

  for (long k0 = kbeg; k0 < kend; k0 += TK) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const long k = k0 + lk + u;
      double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
      if (k < kend) {
        if (aro >= 0) {
          a = A[aro + (ak ? ak[k] : k)];
          if (conjA) a.y = -a.y;
        }
        if (bro >= 0) {
          b = B[bro + (bk ? bk[k] : k)];
          if (conjB) b.y = -b.y;
        }
      }
      As[lk + u][lr] = a;
      Bs[lk + u][lr] = b;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = cfma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }

#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const long m = m0 + ty + 16 * i;
    if (m >= M) continue;
    const long co = cm ? cm[m] : m * ldc;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long n = n0 + tx + 16 * j;
      if (n >= N) continue;
      const long off = co + (cn ? cn[n] : n);
      const double2 x = cmul(alpha, acc[i][j]);
      if (atomic) {
        atomicAdd(&C[off].x, x.x);
        atomicAdd(&C[off].y, x.y);
      } else if (beta.x == 0.0 && beta.y == 0.0) {
        C[off] = x;
      } else {
        C[off] = cadd(x, cmul(beta, C[off]));
      }
    }
  }
}

// y(n) = alpha sum_k A(k) B(n, k) + beta y(n): one thread per output n, the
// loop over k walks each thread's own row (L1 absorbs the stride).
__global__ void gemv_kernel(long N, long K, const double2 *__restrict__ A, const long *__restrict__ ak,
                            bool conjA, const double2 *__restrict__ B, const long *__restrict__ bn,
                            const long *__restrict__ bk, long ldb, bool conjB, double2 *C,
                            const long *__restrict__ cn, long ldc, double2 alpha, double2 beta) {
  for (long n = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; n < N;
       n += static_cast<long>(gridDim.x) * blockDim.x) {
    const long bo = bn ? bn[n] : n * ldb;
    double2 acc[4] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0), make_double2(0.0, 0.0),
                      make_double2(0.0, 0.0)};
    long k = 0;
    for (; k + 4 <= K; k += 4) {  // four independent loads in flight
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        double2 a = A[ak ? ak[k + u] : k + u];
        double2 b = B[bo + (bk ? bk[k + u] : k + u)];
        if (conjA) a.y = -a.y;
        if (conjB) b.y = -b.y;
        acc[u] = cfma(a, b, acc[u]);
      }
    }
    for (; k < K; ++k) {
      double2 a = A[ak ? ak[k] : k];
      double2 b = B[bo + (bk ? bk[k] : k)];
      if (conjA) a.y = -a.y;
      if (conjB) b.y = -b.y;
      acc[0] = cfma(a, b, acc[0]);
    }
    const double2 accs = cadd(cadd(acc[0], acc[1]), cadd(acc[2], acc[3]));
    const long off = cn ? cn[n] : n * ldc;
    const double2 x = cmul(alpha, accs);
    C[off] = (beta.x == 0.0 && beta.y == 0.0) ? x : cadd(x, cmul(beta, C[off]));
  }
}

// Thread-per-output with the K range split over 8 thread rows of the block
// (blockDim 32 x 8) and summed through shared memory: 8x the loads in
// flight of gemv_kernel for long K with a strided operand.
// F32 (tensor-core tiers): products and runs of 16 sums in FP32 on operands
// narrowed on the integer pipes, each run then added in FP64.
__device__ __forceinline__ void cfma32(double2 a, double2 b, bool ca, bool cb, float &xr, float &xi) {
  const float ar = f64_to_f32(a.x), br = f64_to_f32(b.x);
  const float ai = ca ? -f64_to_f32(a.y) : f64_to_f32(a.y);
  const float bi = cb ? -f64_to_f32(b.y) : f64_to_f32(b.y);
  xr = fmaf(ar, br, fmaf(-ai, bi, xr));
  xi = fmaf(ar, bi, fmaf(ai, br, xi));
}

template <bool F32>
__global__ void gemv_kt_kernel(long N, long K, const double2 *__restrict__ A,
                               const long *__restrict__ ak, bool conjA,
                               const double2 *__restrict__ B, const long *__restrict__ bn,
                               const long *__restrict__ bk, long ldb, bool conjB, double2 *C,
                               const long *__restrict__ cn, long ldc, double2 alpha, double2 beta) {
  __shared__ double2 red[8][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const long n = blockIdx.x * 32L + tx;
  double2 acc = make_double2(0.0, 0.0);
  if (n < N) {
    const long bo = bn ? bn[n] : n * ldb;
    // four loads per thread in flight; the sums keep their sequential order
    if (F32) {
      for (long k0 = ty; k0 < K; k0 += 8 * 16) {
        float xr = 0.f, xi = 0.f;
        const long k1 = min(K, k0 + 8 * 16);
        long k = k0;
        for (; k + 24 < k1; k += 32) {
          double2 a[4], b[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const long kk = k + 8 * u;
            a[u] = A[ak ? ak[kk] : kk];
            b[u] = B[bo + (bk ? bk[kk] : kk)];
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) cfma32(a[u], b[u], conjA, conjB, xr, xi);
        }
        for (; k < k1; k += 8)
          cfma32(A[ak ? ak[k] : k], B[bo + (bk ? bk[k] : k)], conjA, conjB, xr, xi);
        acc.x += f32_to_f64(xr);
        acc.y += f32_to_f64(xi);
      }
    } else {
      long k = ty;
      for (; k + 24 < K; k += 32) {
        double2 a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const long kk = k + 8 * u;
          a[u] = A[ak ? ak[kk] : kk];
          b[u] = B[bo + (bk ? bk[kk] : kk)];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (conjA) a[u].y = -a[u].y;
          if (conjB) b[u].y = -b[u].y;
          acc = cfma(a[u], b[u], acc);
        }
      }
      for (; k < K; k += 8) {
        double2 a = A[ak ? ak[k] : k];
        double2 b = B[bo + (bk ? bk[k] : k)];
        if (conjA) a.y = -a.y;
        if (conjB) b.y = -b.y;
        acc = cfma(a, b, acc);
      }
    }
  }
  red[ty][tx] = acc;
  __syncthreads();
  if (ty == 0 && n < N) {
    double2 s = red[0][tx];
#pragma unroll
    for (int y = 1; y < 8; ++y) s = cadd(s, red[y][tx]);
    const long off = cn ? cn[n] : n * ldc;
    const double2 x = cmul(alpha, s);
    C[off] = (beta.x == 0.0 && beta.y == 0.0) ? x : cadd(x, cmul(beta, C[off]));
  }
}

// Same contraction with one warp per output element and the lanes striding
// k: coalesced when the operand's innermost K index has unit stride.
template <bool F32>
__global__ void gemv_warp_kernel(long N, long K, const double2 *__restrict__ A,
                                 const long *__restrict__ ak, bool conjA,
                                 const double2 *__restrict__ B, const long *__restrict__ bn,
                                 const long *__restrict__ bk, long ldb, bool conjB, double2 *C,
                                 const long *__restrict__ cn, long ldc, double2 alpha,
                                 double2 beta) {
  const int lane = threadIdx.x & 31;
  const long wpb = blockDim.x >> 5;
  for (long n = blockIdx.x * wpb + (threadIdx.x >> 5); n < N; n += static_cast<long>(gridDim.x) * wpb) {
    const long bo = bn ? bn[n] : n * ldb;
    // four independent loads per lane in flight (offset tables resolve first)
    double2 ac[4] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0), make_double2(0.0, 0.0),
                     make_double2(0.0, 0.0)};
    long k = lane;
    if (F32) {
      // runs of 4 x 4 products per lane in FP32, each run added in FP64
      for (; k + 96 < K; k += 128) {
        float xr = 0.f, xi = 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const long kk = k + 32 * u;
          cfma32(A[ak ? ak[kk] : kk], B[bo + (bk ? bk[kk] : kk)], conjA, conjB, xr, xi);
        }
        ac[0].x += f32_to_f64(xr);
        ac[0].y += f32_to_f64(xi);
      }
    }
    for (; k + 96 < K; k += 128) {
      long ia[4], ib[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        ia[u] = ak ? ak[k + 32 * u] : k + 32 * u;
        ib[u] = bo + (bk ? bk[k + 32 * u] : k + 32 * u);
      }
      double2 a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = A[ia[u]];
        b[u] = B[ib[u]];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (conjA) a[u].y = -a[u].y;
        if (conjB) b[u].y = -b[u].y;
        ac[u] = cfma(a[u], b[u], ac[u]);
      }
    }
    for (; k < K; k += 32) {
      double2 a = A[ak ? ak[k] : k];
      double2 b = B[bo + (bk ? bk[k] : k)];
      if (conjA) a.y = -a.y;
      if (conjB) b.y = -b.y;
      ac[0] = cfma(a, b, ac[0]);
    }
    double2 acc = cadd(cadd(ac[0], ac[1]), cadd(ac[2], ac[3]));
    for (int o = 16; o > 0; o >>= 1) {
      acc.x += __shfl_down_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_down_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) {
      const long off = cn ? cn[n] : n * ldc;
      const double2 x = cmul(alpha, acc);
      C[off] = (beta.x == 0.0 && beta.y == 0.0) ? x : cadd(x, cmul(beta, C[off]));
    }
  }
}

// Outputs too few to fill the GPU with 64 x 64 tiles (Davidson subspace
// overlaps, the singles intermediates): one warp per output element and a K
// range per blockIdx.y; partial sums are added atomically when K is split (C
// scaled by beta beforehand). F32: runs of four products per lane in FP32,
// each run added in FP64, as in gemv_warp_kernel.
template <bool F32>
__global__ void __launch_bounds__(256) dots_kernel(long M, long N, long K,
                                                   const double2 *__restrict__ A,
                                                   const long *__restrict__ am,
                                                   const long *__restrict__ ak, long lda, bool conjA,
                                                   const double2 *__restrict__ B,
                                                   const long *__restrict__ bn,
                                                   const long *__restrict__ bk, long ldb, bool conjB,
                                                   double2 *C, const long *__restrict__ cm,
                                                   const long *__restrict__ cn, long ldc,
                                                   double2 alpha, double2 beta, long kchunk,
                                                   bool atomic) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long p = blockIdx.x * 8L + warp;
  if (p >= M * N) return;
  const long m = p / N, n = p - m * N;
  const long k0 = blockIdx.y * kchunk, k1 = min(K, k0 + kchunk);
  const long ao = am ? am[m] : m * lda, bo = bn ? bn[n] : n * ldb;
  double2 ac[4] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0), make_double2(0.0, 0.0),
                   make_double2(0.0, 0.0)};
  long k = k0 + lane;
  if (F32) {
    for (; k + 96 < k1; k += 128) {
      float xr = 0.f, xi = 0.f;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long kk = k + 32 * u;
        cfma32(A[ao + (ak ? ak[kk] : kk)], B[bo + (bk ? bk[kk] : kk)], conjA, conjB, xr, xi);
      }
      ac[0].x += f32_to_f64(xr);
      ac[0].y += f32_to_f64(xi);
    }
  }
  for (; k + 96 < k1; k += 128) {
    double2 a[4], b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long kk = k + 32 * u;
      a[u] = A[ao + (ak ? ak[kk] : kk)];
      b[u] = B[bo + (bk ? bk[kk] : kk)];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (conjA) a[u].y = -a[u].y;
      if (conjB) b[u].y = -b[u].y;
      ac[u] = cfma(a[u], b[u], ac[u]);
    }
  }
  for (; k < k1; k += 32) {
    double2 a = A[ao + (ak ? ak[k] : k)], b = B[bo + (bk ? bk[k] : k)];
    if (conjA) a.y = -a.y;
    if (conjB) b.y = -b.y;
    ac[0] = cfma(a, b, ac[0]);
  }
  double2 acc = cadd(cadd(ac[0], ac[1]), cadd(ac[2], ac[3]));
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_down_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_down_sync(0xffffffffu, acc.y, o);
  }
  if (lane == 0) {
    const long off = (cm ? cm[m] : m * ldc) + (cn ? cn[n] : n);
    const double2 x = cmul(alpha, acc);
    if (atomic) {
      atomicAdd(&C[off].x, x.x);
      atomicAdd(&C[off].y, x.y);
    } else {
      C[off] = (beta.x == 0.0 && beta.y == 0.0) ? x : cadd(x, cmul(beta, C[off]));
    }
  }
}

}  // namespace

void gemm_f64(const GemmDesc &g, cudaStream_t st, int num_sms) {
  if (g.M <= 0 || g.N <= 0) return;
  if (g.K <= 0) {
    scale_2d(g.C, g.cm, g.cn, g.ldc, g.M, g.N, g.beta, st);
    return;
  }
  // Matrix-vector shapes are memory bound: one thread per output element.
  // Taken when the vector side and the output's other index need no table
  // (always the case for the engine's size-1 index sets).
  const bool rowvec = g.M == 1 && !g.am && !g.cm;
  const bool colvec = !rowvec && g.N == 1 && !g.bn && !g.cn;
  if (rowvec || colvec) {
    const long n_out = rowvec ? g.N : g.M;
    if (g.k_contig) {
      const unsigned wb = static_cast<unsigned>(std::min<long>((n_out + 7) / 8, 65535));
      auto kern = g.f32 ? gemv_warp_kernel<true> : gemv_warp_kernel<false>;
      if (rowvec)
        kern<<<wb, 256, 0, st>>>(n_out, g.K, g.A, g.ak, g.conjA, g.B, g.bn, g.bk, g.ldb, g.conjB,
                                 g.C, g.cn, 1, g.alpha, g.beta);
      else
        kern<<<wb, 256, 0, st>>>(n_out, g.K, g.B, g.bk, g.conjB, g.A, g.am, g.ak, g.lda, g.conjA,
                                 g.C, g.cm, g.ldc, g.alpha, g.beta);
      LAUNCH_CHECK();
      count_launch();
      return;
    }
    if (g.K >= 64 && n_out <= 65535L * 32) {
      const unsigned kb = static_cast<unsigned>((n_out + 31) / 32);
      auto kern = g.f32 ? gemv_kt_kernel<true> : gemv_kt_kernel<false>;
      if (rowvec)
        kern<<<kb, dim3(32, 8), 0, st>>>(n_out, g.K, g.A, g.ak, g.conjA, g.B, g.bn, g.bk, g.ldb,
                                         g.conjB, g.C, g.cn, 1, g.alpha, g.beta);
      else
        kern<<<kb, dim3(32, 8), 0, st>>>(n_out, g.K, g.B, g.bk, g.conjB, g.A, g.am, g.ak, g.lda,
                                         g.conjA, g.C, g.cm, g.ldc, g.alpha, g.beta);
      LAUNCH_CHECK();
      count_launch();
      return;
    }
    const unsigned blocks = static_cast<unsigned>(std::min<long>((n_out + 255) / 256, 65535));
    if (rowvec) {
      gemv_kernel<<<blocks, 256, 0, st>>>(n_out, g.K, g.A, g.ak, g.conjA, g.B, g.bn, g.bk, g.ldb,
                                          g.conjB, g.C, g.cn, 1, g.alpha, g.beta);
    } else {
      gemv_kernel<<<blocks, 256, 0, st>>>(n_out, g.K, g.B, g.bk, g.conjB, g.A, g.am, g.ak, g.lda,
                                          g.conjA, g.C, g.cm, g.ldc, g.alpha, g.beta);
    }
    LAUNCH_CHECK();
    count_launch();
    return;
  }
  // short K with one short side: FP64 skinny kernel (no tile padding)
  if (g.K <= SKINNY64_MAX_K && std::min(g.M, g.N) <= 256 && std::max(g.M, g.N) >= 1024) {
    SkinnyDesc d;
    d.f64 = true;
    d.K = static_cast<int>(g.K);
    d.alpha = g.alpha;
    d.beta = g.beta;
    d.C = g.C;
    if (g.N <= g.M) {
      d.Mb = g.M; d.Ns = static_cast<int>(g.N);
      d.G = g.A; d.gr = g.am; d.ldg = g.lda; d.gk = g.ak; d.conjG = g.conjA;
      d.S = g.B; d.sr = g.bn; d.lds = g.ldb; d.sk = g.bk; d.conjS = g.conjB;
      d.cb = g.cm; d.ldcb = g.ldc; d.cs = g.cn; d.ldcs = 1;
    } else {
      d.Mb = g.N; d.Ns = static_cast<int>(g.M);
      d.G = g.B; d.gr = g.bn; d.ldg = g.ldb; d.gk = g.bk; d.conjG = g.conjB;
      d.S = g.A; d.sr = g.am; d.lds = g.lda; d.sk = g.ak; d.conjS = g.conjA;
      d.cb = g.cn; d.ldcb = 1; d.cs = g.cm; d.ldcs = g.ldc;
    }
    gemm_skinny(d, st);
    return;
  }
  // Outputs that would leave most SMs without a 64 x 64 tile: one warp per
  // output, K split over blocks until about four blocks per SM. GB300's FP64
  // pipe is narrow (a few FP64 FMAs per clock per SM), so a product on a
  // handful of tiles would run on a handful of SMs.
  const long tiles = ((g.M + TM - 1) / TM) * ((g.N + TN - 1) / TN);
  if (tiles < num_sms && g.M * g.N <= 65535L * 8 && (g.K >= 32 || g.M * g.N <= 4096)) {
    const long gx = (g.M * g.N + 7) / 8;
    long split = std::max<long>(1, std::min<long>(g.K / 256, (4L * num_sms + gx - 1) / gx));
    const long kchunk = (g.K + split - 1) / split;
    split = (g.K + kchunk - 1) / kchunk;
    const bool atomic = split > 1;
    if (atomic) scale_2d(g.C, g.cm, g.cn, g.ldc, g.M, g.N, g.beta, st);
    dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>(split));
    auto kern = g.f32 ? dots_kernel<true> : dots_kernel<false>;
    kern<<<grid, 256, 0, st>>>(g.M, g.N, g.K, g.A, g.am, g.ak, g.lda, g.conjA, g.B, g.bn, g.bk,
                               g.ldb, g.conjB, g.C, g.cm, g.cn, g.ldc, g.alpha, g.beta, kchunk,
                               atomic);
    LAUNCH_CHECK();
    count_launch();
    return;
  }
  long split = 1;
  const long target = 2L * num_sms;
  if (tiles < target && g.K >= 4 * TK * 16) {
    split = std::min<long>((target + tiles - 1) / tiles, (g.K + 255) / 256);
    split = std::max<long>(split, 1);
  }
  long kps = (g.K + split - 1) / split;
  kps = (kps + TK - 1) / TK * TK;
  split = (g.K + kps - 1) / kps;
  const bool atomic = split > 1;
  if (atomic) scale_2d(g.C, g.cm, g.cn, g.ldc, g.M, g.N, g.beta, st);
  dim3 grid(static_cast<unsigned>((g.N + TN - 1) / TN), static_cast<unsigned>((g.M + TM - 1) / TM),
            static_cast<unsigned>(split));
  if (grid.y > 65535) fail(CC_ERR_ARG, "gemm_f64: M too large");
  zgemm_kernel<<<grid, 256, 0, st>>>(g.M, g.N, g.K, g.A, g.am, g.ak, g.lda, g.conjA, g.B, g.bn, g.bk,
                                     g.ldb, g.conjB, g.C, g.cm, g.cn, g.ldc, g.alpha, g.beta, kps,
                                     atomic);
  LAUNCH_CHECK();
  count_launch();
}

}  // namespace cdfns
