#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>

#include "cc_kernels.h"
#include "kernels.h"

namespace cdfns {

namespace {

inline unsigned grid_for(long n, int threads = 256) {
  return static_cast<unsigned>(std::max<long>(1, std::min<long>((n + threads - 1) / threads, 152L * 64)));
}
#define GRID_STRIDE(i, n) \
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < (n); \
       i += static_cast<long>(gridDim.x) * blockDim.x)

// Sum over a block of 256 threads (deterministic order); the result is in
// thread 0.
__device__ double2 block_sum_cc(double2 v) {
  __shared__ double2 sh[8];
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = l < 8 ? sh[l] : make_double2(0.0, 0.0);
    for (int o = 4; o > 0; o >>= 1) {
      v.x += __shfl_down_sync(0xffffffffu, v.x, o);
      v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
  }
  return v;
}

// Row-major pair index of (i < j) among n items and its inverse.
__host__ __device__ inline long pair_index(long i, long j, long n) {
  return i * (2 * n - i - 1) / 2 + (j - i - 1);
}
__device__ inline void pair_decode(long p, long n, int *pi, int *pj) {
  const double b = 2.0 * n - 1.0;
  long i = static_cast<long>(floor((b - sqrt(b * b - 8.0 * static_cast<double>(p))) * 0.5));
  if (i < 0) i = 0;
  while (i > 0 && pair_index(i, i + 1, n) > p) --i;
  while (i + 1 < n - 1 && pair_index(i + 1, i + 2, n) <= p) ++i;
  *pi = static_cast<int>(i);
  *pj = static_cast<int>(p - pair_index(i, i + 1, n) + i + 1);
}

__device__ inline void atomic_max_nonneg(unsigned long long *addr, double x) {
  atomicMax(addr, static_cast<unsigned long long>(__double_as_longlong(x)));
}

__global__ void split_kernel(const double2 *chunk, int np, int p0, int o, int v, double2 *Loo,
                             double2 *Lov, double2 *Lvo, double2 *Lvv, unsigned long long *stats) {
  const int n = o + v;
  const long total = static_cast<long>(np) * n * n;
  double mx = 0.0, asym = 0.0;
  unsigned long long bad = 0;
  GRID_STRIDE(idx, total) {
    const int P = static_cast<int>(idx / (static_cast<long>(n) * n));
    const int p = static_cast<int>((idx / n) % n);
    const int q = static_cast<int>(idx % n);
    const double2 x = chunk[idx];
    const double2 y = chunk[(static_cast<long>(P) * n + q) * n + p];
    if (!isfinite(x.x) || !isfinite(x.y)) ++bad;
    mx = fmax(mx, fmax(fabs(x.x), fabs(x.y)));
    asym = fmax(asym, fmax(fabs(x.x - y.x), fabs(x.y + y.y)));
    const long PP = p0 + P;
    // a NULL destination block is skipped (streamed natural spinors)
    if (p < o && q < o) {
      if (Loo) Loo[(PP * o + p) * o + q] = x;
    } else if (p < o) {
      if (Lov) Lov[(PP * o + p) * v + (q - o)] = x;
    } else if (q < o) {
      if (Lvo) Lvo[(PP * v + (p - o)) * o + q] = x;
    } else if (Lvv) {
      Lvv[(PP * v + (p - o)) * v + (q - o)] = x;
    }
  }
  for (int s = 16; s > 0; s >>= 1) {
    mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, s));
    asym = fmax(asym, __shfl_down_sync(0xffffffffu, asym, s));
    bad += __shfl_down_sync(0xffffffffu, bad, s);
  }
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(&stats[0], mx);
    atomic_max_nonneg(&stats[1], asym);
    if (bad) atomicAdd(&stats[2], bad);
  }
}

// Elementwise kernels over [o][o][v][v] use a 2D grid: blockIdx.y walks the
// (i, j) planes, threads walk (a, b) inside a plane (32-bit index math).
// Doubles-sized forms built from t2 and a product of two t1 rows. One block
// per (i, j) and 32 rows a; the rows t1[i][:], t1[j][:] sit in shared memory.
//   ANTI: x_ab = t_ia t_jb - t_ib t_ja (tau), else x_ab = t_ia t_jb (Z)
//   out0 = c0 t2 + f0 x, and out1 = t2 + f1 x when out1 is given.
// F32 (tensor-core tiers, whose GEMMs round these operands to TF32/BF16 or
// split them at FP32 level): the t1 products in FP32, converted on the
// integer pipes, so each element costs only its FP64 additions.
template <typename R>
struct RowT;
template <>
struct RowT<float2> {
  __device__ static float2 load(double2 x) { return make_float2(f64_to_f32(x.x), f64_to_f32(x.y)); }
};
template <>
struct RowT<double2> {
  __device__ static double2 load(double2 x) { return x; }
};

__device__ __forceinline__ float2 tmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 tmul(double2 a, double2 b) { return cmul(a, b); }
__device__ __forceinline__ float2 tsub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 tsub(double2 a, double2 b) { return csub(a, b); }
__device__ __forceinline__ double2 widen_scaled(float2 x, float f) {
  return make_double2(f32_to_f64(f * x.x), f32_to_f64(f * x.y));
}
__device__ __forceinline__ double2 widen_scaled(double2 x, float f) { return cscale(f, x); }

// exact c * x for c in {1, 1/2}: the halving lowers the exponent of a normal
// number (integer pipes); zeros and values near the bottom of the range use
// the FP64 multiply
__device__ __forceinline__ double scale_c(double x, int half) {
  if (!half) return x;
  const long long b = __double_as_longlong(x);
  const unsigned e = static_cast<unsigned>(b >> 52) & 0x7ffu;
  if (e - 2u <= 0x7feu - 2u) return __longlong_as_double(b - (1LL << 52));
  if ((static_cast<unsigned long long>(b) << 1) == 0ull) return x;
  return 0.5 * x;
}

// max(|Re|, |Im|) in FP32 of one complex value (the FP16 tiers' scale source)
__device__ __forceinline__ float mag32(double2 x) {
  return fmaxf(fabsf(f64_to_f32(x.x)), fabsf(f64_to_f32(x.y)));
}

// Block maxima of three values combined into mx[0..2] (device floats, zeroed
// by the caller) with unsigned atomicMax on the float bits; a block skips the
// atomic when the stored value is already as large (the maximum only grows,
// so a stale read costs an extra atomic, never a wrong result).
__device__ __forceinline__ void block_max3(float m0, float m1, float m2, float *mx) {
  __shared__ float sh[3][8];
  for (int s = 16; s > 0; s >>= 1) {
    m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, s));
    m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, s));
    m2 = fmaxf(m2, __shfl_xor_sync(0xffffffffu, m2, s));
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sh[0][w] = m0;
    sh[1][w] = m1;
    sh[2][w] = m2;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    float x = 0.0f;
    for (int i = 0; i < static_cast<int>(blockDim.x >> 5); ++i) x = fmaxf(x, sh[threadIdx.x][i]);
    unsigned *dst = reinterpret_cast<unsigned *>(mx + threadIdx.x);
    if (__float_as_uint(x) > *reinterpret_cast<volatile unsigned *>(dst))
      atomicMax(dst, __float_as_uint(x));
  }
}

// mx (optional, three zeroed device floats): the maxima of t2, out0 and out1
// over the whole tensors, for the FP16 tiers' operand scales.
template <typename T, bool ANTI>
__global__ void __launch_bounds__(256) t1t1_kernel(const double2 *__restrict__ t1,
                                                   const double2 *__restrict__ t2, double2 *out0,
                                                   double2 *out1, int o, int v, int c0_half,
                                                   double c0, float f0, float f1, float *mx) {
  extern __shared__ __align__(16) unsigned char t1t1_sm[];
  T *ti = reinterpret_cast<T *>(t1t1_sm);
  T *tj = ti + v;
  const int ij = blockIdx.y;
  const int i = ij / o, j = ij - (ij / o) * o;
  for (int b = threadIdx.x; b < v; b += blockDim.x) {
    ti[b] = RowT<T>::load(t1[static_cast<long>(i) * v + b]);
    tj[b] = RowT<T>::load(t1[static_cast<long>(j) * v + b]);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long base = static_cast<long>(ij) * v * v;
  const int a_end = min(v, static_cast<int>(blockIdx.x) * 32 + 32);
  float m_t = 0.0f, m_0 = 0.0f, m_1 = 0.0f;
  for (int a = blockIdx.x * 32 + warp; a < a_end; a += 8) {
    const T tia = ti[a], tja = tj[a];
    const long row = base + static_cast<long>(a) * v;
    for (int b = lane; b < v; b += 32) {
      T x = tmul(tia, tj[b]);
      if (ANTI) x = tsub(x, tmul(ti[b], tja));
      const double2 t = t2[row + b];
      const double2 p0 = widen_scaled(x, f0);
      double2 r0;
      if (c0_half >= 0) {
        r0 = make_double2(scale_c(t.x, c0_half) + p0.x, scale_c(t.y, c0_half) + p0.y);
      } else {
        r0 = make_double2(c0 * t.x + p0.x, c0 * t.y + p0.y);
      }
      out0[row + b] = r0;
      if (mx) {
        m_t = fmaxf(m_t, mag32(t));
        m_0 = fmaxf(m_0, mag32(r0));
      }
      if (out1) {
        const double2 p1 = widen_scaled(x, f1);
        const double2 r1 = make_double2(t.x + p1.x, t.y + p1.y);
        out1[row + b] = r1;
        if (mx) m_1 = fmaxf(m_1, mag32(r1));
      }
    }
  }
  if (mx) block_max3(m_t, m_0, m_1, mx);
}


__global__ void jacobi_kernel(const double2 *R1, const double2 *R2, const double *eps, int o, int v,
                              double2 *t1, double2 *t2) {
  const int vv = v * v;
  for (int ij = blockIdx.y; ij < o * o; ij += gridDim.y) {
    const int i = ij / o, j = ij - (ij / o) * o;
    const long base = static_cast<long>(ij) * vv;
    const double eij = eps[i] + eps[j];
    for (int ab = blockIdx.x * blockDim.x + threadIdx.x; ab < vv; ab += gridDim.x * blockDim.x) {
      const int a = ab / v, b = ab - (ab / v) * v;
      if (i == j || a == b) {
        t2[base + ab] = make_double2(0.0, 0.0);
      } else {
        const double inv = 1.0 / (eij - eps[o + a] - eps[o + b]);
        const double2 r = R2[base + ab];
        t2[base + ab] = make_double2(r.x * inv, r.y * inv);
      }
      if (ij == 0 && ab < o * v) {
        const int ii = ab / v, aa = ab - (ab / v) * v;
        const double d = eps[ii] - eps[o + aa];
        t1[ab] = make_double2(R1[ab].x / d, R1[ab].y / d);
      }
    }
  }
}

__global__ void mp2_kernel(const double2 *oovv, const double *eps, int o, int v, double2 *t1,
                           double2 *t2) {
  const long n1 = static_cast<long>(o) * v;
  const long total = static_cast<long>(o) * o * v * v;
  GRID_STRIDE(idx, total) {
    const int b = static_cast<int>(idx % v);
    const int a = static_cast<int>((idx / v) % v);
    const int j = static_cast<int>((idx / (static_cast<long>(v) * v)) % o);
    const int i = static_cast<int>(idx / (static_cast<long>(v) * v * o));
    if (i == j || a == b) {
      t2[idx] = make_double2(0.0, 0.0);
    } else {
      const double d = eps[i] + eps[j] - eps[o + a] - eps[o + b];
      t2[idx] = make_double2(oovv[idx].x / d, -oovv[idx].y / d);
    }
    if (idx < n1) t1[idx] = make_double2(0.0, 0.0);
  }
}

__global__ void pack_amps_kernel(const double2 *t1, const double2 *t2, int o, int v,
                                 const int *ij_i, const int *ij_j, const int *ab_a,
                                 const int *ab_b, double2 *vec) {
  const long n1 = static_cast<long>(o) * v;
  const long nab = static_cast<long>(v) * (v - 1) / 2;
  const long nij = static_cast<long>(o) * (o - 1) / 2;
  const long total = n1 + nij * nab;
  GRID_STRIDE(idx, total) {
    if (idx < n1) {
      vec[idx] = t1[idx];
    } else {
      const long q = idx - n1;
      const long pij = q / nab, pab = q - (q / nab) * nab;
      const int i = ij_i[pij], j = ij_j[pij], a = ab_a[pab], b = ab_b[pab];
      vec[idx] = t2[((static_cast<long>(i) * o + j) * v + a) * v + b];
    }
  }
}

// Full t1, t2 from the packed unique amplitudes. Block: one (i, j) row and
// 8 rows a; lanes run along b. The four images of a unique element differ
// by sign only, applied to the sign bits.
__device__ __forceinline__ double2 neg_if(double2 x, bool neg) {
  if (!neg) return x;
  return make_double2(__longlong_as_double(__double_as_longlong(x.x) ^ (1LL << 63)),
                      __longlong_as_double(__double_as_longlong(x.y) ^ (1LL << 63)));
}

__global__ void __launch_bounds__(256) unpack_amps_kernel(const double2 *__restrict__ vec, int o,
                                                          int v, double2 *t1, double2 *t2) {
  const long n1 = static_cast<long>(o) * v;
  const long nab = static_cast<long>(v) * (v - 1) / 2;
  const int ij = blockIdx.y;
  const int i = ij / o, j = ij - (ij / o) * o;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int a = blockIdx.x * 8 + warp;
  if (blockIdx.x == 0 && ij == 0)
    for (long k = threadIdx.x; k < n1; k += blockDim.x) t1[k] = vec[k];
  if (a >= v) return;
  double2 *out = t2 + (static_cast<long>(ij) * v + a) * v;
  if (i == j) {
    for (int b = lane; b < v; b += 32) out[b] = make_double2(0.0, 0.0);
    return;
  }
  const int ii = min(i, j), jj = max(i, j);
  const double2 *row = vec + n1 + pair_index(ii, jj, o) * nab;
  for (int b = lane; b < v; b += 32) {
    double2 x = make_double2(0.0, 0.0);
    if (a != b) {
      const int aa = min(a, b), bb = max(a, b);
      x = neg_if(row[pair_index(aa, bb, v)], (i < j) != (a < b));
    }
    out[b] = x;
  }
}

// 1 / D for every packed amplitude: e_i - e_a (singles), e_i + e_j - e_a -
// e_b (doubles); computed once per solve, in FP64.
__global__ void amp_denoms_kernel(const double *eps, int o, int v, const int *ij_i, const int *ij_j,
                                  const int *ab_a, const int *ab_b, double *inv) {
  const long n1 = static_cast<long>(o) * v;
  const long nab = static_cast<long>(v) * (v - 1) / 2;
  const long nij = static_cast<long>(o) * (o - 1) / 2;
  const long total = n1 + nij * nab;
  GRID_STRIDE(idx, total) {
    double d;
    if (idx < n1) {
      const int i = static_cast<int>(idx / v), a = static_cast<int>(idx - (idx / v) * v);
      d = eps[i] - eps[o + a];
    } else {
      const long q = idx - n1;
      const long pij = q / nab, pab = q - pij * nab;
      d = eps[ij_i[pij]] + eps[ij_j[pij]] - eps[o + ab_a[pab]] - eps[o + ab_b[pab]];
    }
    inv[idx] = 1.0 / d;
  }
}

// Jacobi step straight into the packed vector: vec = R * (1/D) over the
// unique amplitudes. Grid (pab chunks, pij) for the doubles; the first row
// of blocks also does the singles.
__global__ void __launch_bounds__(256) jacobi_packed_kernel(
    const double2 *__restrict__ R1, const double2 *__restrict__ R2, const double *__restrict__ inv,
    int o, int v, const int *__restrict__ ij_i, const int *__restrict__ ij_j,
    const int *__restrict__ ab_a, const int *__restrict__ ab_b, double2 *vec) {
  const long n1 = static_cast<long>(o) * v;
  const long nab = static_cast<long>(v) * (v - 1) / 2;
  const int pij = blockIdx.y;
  if (pij == 0)
    for (long k = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; k < n1;
         k += static_cast<long>(gridDim.x) * blockDim.x) {
      const double2 r = R1[k];
      vec[k] = make_double2(r.x * inv[k], r.y * inv[k]);
    }
  const int i = ij_i[pij], j = ij_j[pij];
  const double2 *Rij = R2 + (static_cast<long>(i) * o + j) * v * v;
  const long base = n1 + pij * nab;
  for (long pab = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; pab < nab;
       pab += static_cast<long>(gridDim.x) * blockDim.x) {
    const double2 r = Rij[static_cast<long>(ab_a[pab]) * v + ab_b[pab]];
    const double w = inv[base + pab];
    vec[base + pab] = make_double2(r.x * w, r.y * w);
  }
}

// E = sum over i<j, a<b of <ij||ab> (t_ij^ab + t_i^a t_j^b - t_i^b t_j^a)
// from the packed amplitudes (Eq. 15 restricted to unique elements: the
// four images of each give the 1/4 and 1/2 prefactors); FP64 sums, block
// partials in partial[blockIdx.y * gridDim.x + blockIdx.x]. F32: the small
// t1 t1 products in FP32.
template <bool F32>
__global__ void __launch_bounds__(256) energy_packed_kernel(
    const double2 *__restrict__ oovv, const double2 *__restrict__ vec, int o, int v,
    const int *__restrict__ ij_i, const int *__restrict__ ij_j, const int *__restrict__ ab_a,
    const int *__restrict__ ab_b, double2 *partial) {
  const long n1 = static_cast<long>(o) * v;
  const long nab = static_cast<long>(v) * (v - 1) / 2;
  const int pij = blockIdx.y;
  const int i = ij_i[pij], j = ij_j[pij];
  const double2 *g = oovv + (static_cast<long>(i) * o + j) * v * v;
  const double2 *tp = vec + n1 + pij * nab;
  const double2 *ti = vec + static_cast<long>(i) * v, *tj = vec + static_cast<long>(j) * v;
  double2 acc = make_double2(0.0, 0.0);
  for (long pab = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; pab < nab;
       pab += static_cast<long>(gridDim.x) * blockDim.x) {
    const int a = ab_a[pab], b = ab_b[pab];
    double2 tau = tp[pab];
    if (F32) {
      const double2 p = ti[a], q = tj[b], r = ti[b], u = tj[a];
      const float px = f64_to_f32(p.x), py = f64_to_f32(p.y), qx = f64_to_f32(q.x),
                  qy = f64_to_f32(q.y), rx = f64_to_f32(r.x), ry = f64_to_f32(r.y),
                  ux = f64_to_f32(u.x), uy = f64_to_f32(u.y);
      tau.x += f32_to_f64((px * qx - py * qy) - (rx * ux - ry * uy));
      tau.y += f32_to_f64((px * qy + py * qx) - (rx * uy + ry * ux));
    } else {
      tau = cadd(tau, csub(cmul(ti[a], tj[b]), cmul(ti[b], tj[a])));
    }
    acc = cfma(g[static_cast<long>(a) * v + b], tau, acc);
  }
  acc = block_sum_cc(acc);
  if (threadIdx.x == 0) partial[static_cast<long>(blockIdx.y) * gridDim.x + blockIdx.x] = acc;
}

__global__ void sum_partials_kernel(const double2 *partial, long np, double2 *res) {
  double2 acc = make_double2(0.0, 0.0);
  for (long k = threadIdx.x; k < np; k += blockDim.x) acc = cadd(acc, partial[k]);
  acc = block_sum_cc(acc);
  if (threadIdx.x == 0) *res = acc;
}

__global__ void diis_solve_kernel(const double2 *B, int m, int ldb, double2 *coef, int *status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  constexpr int MX = 17;
  double2 A[MX][MX + 1];
  const int n = m + 1;
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j < m; ++j) A[i][j] = B[i * ldb + j];
    A[i][m] = make_double2(-1.0, 0.0);
    A[i][n] = make_double2(0.0, 0.0);
  }
  for (int j = 0; j < m; ++j) A[m][j] = make_double2(-1.0, 0.0);
  A[m][m] = make_double2(0.0, 0.0);
  A[m][n] = make_double2(-1.0, 0.0);
  // scale rows 0..m-1 / columns by the mean diagonal to keep the pivots sane
  double sc = 0.0;
  for (int i = 0; i < m; ++i) sc += fabs(A[i][i].x);
  sc = sc > 0 ? sc / m : 1.0;
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) A[i][j] = cscale(1.0 / sc, A[i][j]);
  int ok = 0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    double best = hypot(A[c][c].x, A[c][c].y);
    for (int r = c + 1; r < n; ++r) {
      const double x = hypot(A[r][c].x, A[r][c].y);
      if (x > best) { best = x; piv = r; }
    }
    if (best < 1e-300) { ok = 1; break; }
    if (piv != c)
      for (int k = 0; k <= n; ++k) { const double2 t = A[c][k]; A[c][k] = A[piv][k]; A[piv][k] = t; }
    const double2 d = A[c][c];
    const double dd = d.x * d.x + d.y * d.y;
    const double2 inv = make_double2(d.x / dd, -d.y / dd);
    for (int r = c + 1; r < n; ++r) {
      const double2 f = cmul(A[r][c], inv);
      for (int k = c; k <= n; ++k) A[r][k] = csub(A[r][k], cmul(f, A[c][k]));
    }
  }
  if (!ok) {
    double2 x[MX];
    for (int r = n - 1; r >= 0; --r) {
      double2 s = A[r][n];
      for (int k = r + 1; k < n; ++k) s = csub(s, cmul(A[r][k], x[k]));
      const double2 d = A[r][r];
      const double dd = d.x * d.x + d.y * d.y;
      x[r] = cmul(s, make_double2(d.x / dd, -d.y / dd));
    }
    for (int i = 0; i < m; ++i) {
      coef[i] = x[i];
      if (!isfinite(x[i].x) || !isfinite(x[i].y)) ok = 1;
    }
  }
  *status = ok;
}

struct VecPtrs {
  double2 *p[16];
};

__global__ void combine_kernel(VecPtrs vp, const double2 *coef, int m, long n, double2 *out) {
  GRID_STRIDE(i, n) {
    double2 acc = make_double2(0.0, 0.0);
    for (int k = 0; k < m; ++k) acc = cfma(coef[k], vp.p[k][i], acc);
    out[i] = acc;
  }
}

template <int MODE>  // 0: f32 planes, 1: bf16 planes, 2: double2 matrix
__global__ void antisym_kernel(const void *Vp, bool f32, int v, int a0, long p0, long p1,
                               const int *pair_a, const int *pair_b, const int *cd_c,
                               const int *cd_d, long ncd, void *hi, void *lo, long kp,
                               double2 *w64) {
  const long np = p1 - p0;
  const long ld = static_cast<long>(v - a0) * v;
  const long total = np * ncd;
  GRID_STRIDE(idx, total) {
    const long r = idx / ncd, q = idx % ncd;
    const int a = pair_a[p0 + r], b = pair_b[p0 + r];
    const int c = cd_c[q], d = cd_d[q];
    const long ra = static_cast<long>(a - a0) * v, cb = static_cast<long>(b - a0) * v;
    double wr, wi;
    if (f32) {
      const float2 *V = reinterpret_cast<const float2 *>(Vp);
      const float2 x = V[(ra + c) * ld + cb + d];
      const float2 y = V[(ra + d) * ld + cb + c];
      wr = static_cast<double>(x.x) - y.x;
      wi = static_cast<double>(x.y) - y.y;
    } else {
      const double2 *V = reinterpret_cast<const double2 *>(Vp);
      const double2 x = V[(ra + c) * ld + cb + d];
      const double2 y = V[(ra + d) * ld + cb + c];
      wr = x.x - y.x;
      wi = x.y - y.y;
    }
    if (MODE == 2) {
      w64[r * ncd + q] = make_double2(wr, wi);
    } else if (MODE == 0) {
      float *h = reinterpret_cast<float *>(hi);
      float *l = reinterpret_cast<float *>(lo);
      const float fr = static_cast<float>(wr), fi = static_cast<float>(wi);
      uint32_t ur, ui;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(ur) : "f"(fr));
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(ui) : "f"(fi));
      const float hr = __uint_as_float(ur), hi_ = __uint_as_float(ui);
      h[r * kp + 2 * q] = hr;
      h[r * kp + 2 * q + 1] = hi_;
      if (l) {
        uint32_t lr, li;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lr) : "f"(fr - hr));
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(li) : "f"(fi - hi_));
        l[r * kp + 2 * q] = __uint_as_float(lr);
        l[r * kp + 2 * q + 1] = __uint_as_float(li);
      }
    } else {
      __nv_bfloat16 *h = reinterpret_cast<__nv_bfloat16 *>(hi);
      __nv_bfloat16 *l = reinterpret_cast<__nv_bfloat16 *>(lo);
      const float fr = static_cast<float>(wr), fi = static_cast<float>(wi);
      const __nv_bfloat16 hr = __float2bfloat16_rn(fr), hi_ = __float2bfloat16_rn(fi);
      h[r * kp + 2 * q] = hr;
      h[r * kp + 2 * q + 1] = hi_;
      l[r * kp + 2 * q] = __float2bfloat16_rn(fr - __bfloat162float(hr));
      l[r * kp + 2 * q + 1] = __float2bfloat16_rn(fi - __bfloat162float(hi_));
    }
  }
}

// Tensor-core tiers: W[(a,b)][(c<d)] = V[a][c][b][d] - V[a][d][b][c] from the
// FP32 slab. Block (32, 8) per (a, b) pair row and (C <= D) pair of 32-wide
// tiles of c and d: the tiles V[a][C][b][D] and V[a][D][b][C] are read along
// their inner index into shared memory, and W is written along d (packed
// (c<d) columns are contiguous in d for fixed c). Differences in FP32; PT:
// 0 tf32 hi (+ lo), 1 bf16 hi (+ lo), 2 fp16 scaled by fp16_scale(*amax),
// 3 fp16 hi + lo of the scaled value.
template <int PT>
__global__ void __launch_bounds__(256) antisym_tile_kernel(
    const float2 *__restrict__ V, int v, int a0, long p0, long np, const int *__restrict__ pair_a,
    const int *__restrict__ pair_b, void *hi, void *lo, long kp, int ntile, const float *amax) {
  __shared__ float2 s1[32][33];  // V[a][c][b][d], c = C0 + row
  __shared__ float2 s2[32][33];  // V[a][d][b][c], d = D0 + row
  const int tx = threadIdx.x, ty = threadIdx.y;
  int ct = 0, p = blockIdx.x;
  while (p >= ntile - ct) {
    p -= ntile - ct;
    ++ct;
  }
  const int dt = ct + p;
  const int C0 = ct * 32, D0 = dt * 32;
  const long ld = static_cast<long>(v - a0) * v;
  const float sc = (PT >= 2 && amax) ? fp16_scale(*amax) : 1.0f;
  // Each block walks many pairs r; the tiles of the next pair are loaded into
  // registers while the current one is antisymmetrised and stored, so every
  // thread keeps eight loads in flight across the loop.
  float2 n1[4], n2[4];
  auto fetch = [&](long r) {
    const int a = pair_a[p0 + r], b = pair_b[p0 + r];
    const long ra = static_cast<long>(a - a0) * v, cb = static_cast<long>(b - a0) * v;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int row = ty + 8 * j;
      const int c = C0 + row, d = D0 + tx;
      n1[j] = (c < v && d < v) ? V[(ra + c) * ld + cb + d] : make_float2(0.f, 0.f);
      const int d2 = D0 + row, c2 = C0 + tx;
      n2[j] = (d2 < v && c2 < v) ? V[(ra + d2) * ld + cb + c2] : make_float2(0.f, 0.f);
    }
  };
  if (blockIdx.y < np) fetch(blockIdx.y);
  for (long r = blockIdx.y; r < np; r += gridDim.y) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      s1[ty + 8 * j][tx] = n1[j];
      s2[ty + 8 * j][tx] = n2[j];
    }
    __syncthreads();
    if (r + gridDim.y < np) fetch(r + gridDim.y);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int row = ty + 8 * j;
      const int c = C0 + row, d = D0 + tx;
      if (c < d && d < v) {
        const float2 x = s1[row][tx], y = s2[tx][row];
        const float wr = x.x - y.x, wi = x.y - y.y;
        const long q = static_cast<long>(c) * (2L * v - c - 1) / 2 + (d - c - 1);
        const long e = r * kp + 2 * q;  // even: paired stores
        if constexpr (PT == 0) {
          uint32_t ur, ui;
          asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(ur) : "f"(wr));
          asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(ui) : "f"(wi));
          const float hr = __uint_as_float(ur), hi_ = __uint_as_float(ui);
          reinterpret_cast<float2 *>(hi)[e >> 1] = make_float2(hr, hi_);
          if (lo) {
            uint32_t lr, li;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lr) : "f"(wr - hr));
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(li) : "f"(wi - hi_));
            reinterpret_cast<float2 *>(lo)[e >> 1] = make_float2(__uint_as_float(lr), __uint_as_float(li));
          }
        } else if constexpr (PT == 1) {
          const __nv_bfloat162 h = __floats2bfloat162_rn(wr, wi);
          reinterpret_cast<__nv_bfloat162 *>(hi)[e >> 1] = h;
          const float2 hf = __bfloat1622float2(h);
          reinterpret_cast<__nv_bfloat162 *>(lo)[e >> 1] = __floats2bfloat162_rn(wr - hf.x, wi - hf.y);
        } else {
          const float sr = sc * wr, si = sc * wi;
          const __half2 h = __floats2half2_rn(sr, si);
          reinterpret_cast<__half2 *>(hi)[e >> 1] = h;
          if (PT == 3) {
            const float2 hf = __half22float2(h);
            reinterpret_cast<__half2 *>(lo)[e >> 1] = __floats2half2_rn(sr - hf.x, si - hf.y);
          }
        }
      }
    }
    __syncthreads();
  }
}

// zero the padded tail columns [2*ncd, kp) of rows [0, np)
template <typename E>
__global__ void zero_tail(E *p, long np, long k0, long kp) {
  const long w = kp - k0;
  GRID_STRIDE(idx, np * w) {
    const long r = idx / w, k = k0 + idx % w;
    p[r * kp + k] = E(0);
  }
}

__global__ void unpack_pairs_kernel(const double2 *R, int o, int v, const int *ij_i,
                                    const int *ij_j, const int *ab_a, const int *ab_b,
                                    double2 *R2) {
  const long nij = static_cast<long>(o) * (o - 1) / 2;
  const long nab = static_cast<long>(v) * (v - 1) / 2;
  GRID_STRIDE(idx, nij * nab) {
    const long p = idx / nab, q = idx % nab;
    const int i = ij_i[p], j = ij_j[p], a = ab_a[q], b = ab_b[q];
    const double2 x = R[idx];
    const long vv = static_cast<long>(v) * v;
    double2 *e;
    e = &R2[(static_cast<long>(i) * o + j) * vv + static_cast<long>(a) * v + b]; *e = cadd(*e, x);
    e = &R2[(static_cast<long>(j) * o + i) * vv + static_cast<long>(a) * v + b]; *e = csub(*e, x);
    e = &R2[(static_cast<long>(i) * o + j) * vv + static_cast<long>(b) * v + a]; *e = csub(*e, x);
    e = &R2[(static_cast<long>(j) * o + i) * vv + static_cast<long>(b) * v + a]; *e = cadd(*e, x);
  }
}

// Same update, one block (32, 8) per (i<j) pair and (A <= B) pair of 32-wide
// tiles of a and b: the packed values of the tile are read along b into
// shared memory, then R2[ij] and R2[ji] are updated along b at [a][b] and,
// through the transposed tile, along a at [b][a]. Every element of R2 has
// one writer (no atomics) and every access runs along a contiguous index.
__global__ void __launch_bounds__(256) unpack_pairs_tile_kernel(const double2 *__restrict__ R,
                                                                int o, int v,
                                                                const int *__restrict__ ij_i,
                                                                const int *__restrict__ ij_j,
                                                                double2 *R2, int nt) {
  __shared__ double2 s[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  int at = 0, t = blockIdx.x;
  while (t >= nt - at) {
    t -= nt - at;
    ++at;
  }
  const int A0 = at * 32, B0 = (at + t) * 32;
  const long pr = blockIdx.y;
  const long nab = static_cast<long>(v) * (v - 1) / 2;
  const double2 *Rp = R + pr * nab;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int a = A0 + ty + 8 * j, b = B0 + tx;
    double2 x = make_double2(0.0, 0.0);
    if (a < b && b < v) x = Rp[static_cast<long>(a) * (2L * v - a - 1) / 2 + (b - a - 1)];
    s[ty + 8 * j][tx] = x;
  }
  __syncthreads();
  const int i = ij_i[pr], jj = ij_j[pr];
  const long vv = static_cast<long>(v) * v;
  double2 *Rij = R2 + (static_cast<long>(i) * o + jj) * vv;
  double2 *Rji = R2 + (static_cast<long>(jj) * o + i) * vv;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int a = A0 + ty + 8 * j, b = B0 + tx;  // [a][b], a < b: + R(a, b)
    if (a < b && b < v) {
      const double2 x = s[ty + 8 * j][tx];
      const long e = static_cast<long>(a) * v + b;
      Rij[e] = cadd(Rij[e], x);
      Rji[e] = csub(Rji[e], x);
    }
    const int b2 = B0 + ty + 8 * j, a2 = A0 + tx;  // [b2][a2], a2 < b2: - R(a2, b2)
    if (a2 < b2 && b2 < v) {
      const double2 x = s[tx][ty + 8 * j];
      const long e = static_cast<long>(b2) * v + a2;
      Rij[e] = csub(Rij[e], x);
      Rji[e] = cadd(Rji[e], x);
    }
  }
}

__global__ void pairs_kernel(int n, int *pi, int *pj) {
  const long np = static_cast<long>(n) * (n - 1) / 2;
  GRID_STRIDE(p, np) {
    int i, j;
    pair_decode(p, n, &i, &j);
    pi[p] = i;
    pj[p] = j;
  }
}

__global__ void ip_unpack_kernel(const double2 *vec, int k, int o, int v, double2 *r1,
                                 double2 *r2) {
  const long dim = o + static_cast<long>(o) * (o - 1) / 2 * v;
  const long per = static_cast<long>(o) * o * v;
  GRID_STRIDE(idx, static_cast<long>(k) * per) {
    const long kk = idx / per, rem = idx % per;
    const int b = static_cast<int>(rem % v);
    const int j = static_cast<int>((rem / v) % o);
    const int i = static_cast<int>(rem / (static_cast<long>(v) * o));
    double2 x = make_double2(0.0, 0.0);
    if (i < j) x = vec[kk * dim + o + pair_index(i, j, o) * v + b];
    else if (j < i) x = cscale(-1.0, vec[kk * dim + o + pair_index(j, i, o) * v + b]);
    r2[idx] = x;
    if (rem < o) r1[kk * o + rem] = vec[kk * dim + rem];
  }
}

__global__ void ip_pack_kernel(const double2 *r1, const double2 *r2, int k, int o, int v,
                               double2 *vec) {
  const long np = static_cast<long>(o) * (o - 1) / 2;
  const long dim = o + np * v;
  GRID_STRIDE(idx, static_cast<long>(k) * dim) {
    const long kk = idx / dim, rem = idx % dim;
    if (rem < o) {
      vec[idx] = r1[kk * o + rem];
    } else {
      const long q = rem - o;
      int i, j;
      pair_decode(q / v, o, &i, &j);
      const int b = static_cast<int>(q % v);
      vec[idx] = r2[((kk * o + i) * o + j) * v + b];
    }
  }
}

__global__ void ip_diag_kernel(const double2 *Hoo, const double2 *Hvv, int o, int v, double2 *d) {
  const long np = static_cast<long>(o) * (o - 1) / 2;
  const long dim = o + np * v;
  GRID_STRIDE(idx, dim) {
    if (idx < o) {
      d[idx] = cscale(-1.0, Hoo[idx * o + idx]);
    } else {
      const long q = idx - o;
      int i, j;
      pair_decode(q / v, o, &i, &j);
      const int b = static_cast<int>(q % v);
      d[idx] = csub(csub(Hvv[static_cast<long>(b) * v + b], Hoo[static_cast<long>(i) * o + i]),
                    Hoo[static_cast<long>(j) * o + j]);
    }
  }
}

__global__ void ip_diag_apply_kernel(const double2 *r1, const double2 *r2, const double2 *doo,
                                     const double2 *dvv, int k, int o, int v, double2 *s1,
                                     double2 *s2) {
  const long per = static_cast<long>(o) * o * v;
  GRID_STRIDE(idx, static_cast<long>(k) * per) {
    const long kk = idx / per, rem = idx % per;
    const int b = static_cast<int>(rem % v);
    const int j = static_cast<int>((rem / v) % o);
    const int i = static_cast<int>(rem / (static_cast<long>(v) * o));
    const double2 d = csub(csub(dvv[b], doo[i]), doo[j]);
    s2[idx] = cadd(s2[idx], cmul(d, r2[idx]));
    if (rem < o) s1[kk * o + rem] = csub(s1[kk * o + rem], cmul(doo[rem], r1[kk * o + rem]));
  }
}

// s2 += tA + tB + tC - P(ij) X1 + P(ij) X2 on [k][o][o][v] tensors
__global__ void sigma_combine_kernel(double2 *s2, const double2 *tA, const double2 *tB,
                                     const double2 *tC, const double2 *X1, const double2 *X2, int k,
                                     int o, int v) {
  const long per = static_cast<long>(o) * o * v;
  GRID_STRIDE(idx, static_cast<long>(k) * per) {
    const long kk = idx / per, rem = idx % per;
    const int b = static_cast<int>(rem % v);
    const int j = static_cast<int>((rem / v) % o);
    const int i = static_cast<int>(rem / (static_cast<long>(v) * o));
    const long sw = kk * per + (static_cast<long>(j) * o + i) * v + b;
    double2 x = cadd(cadd(s2[idx], tA[idx]), cadd(tB[idx], tC[idx]));
    x = cadd(x, csub(X1[sw], X1[idx]));
    x = cadd(x, csub(X2[idx], X2[sw]));
    s2[idx] = x;
  }
}

__global__ void split_diag_kernel(const double2 *A, int n, double2 *off, double2 *diag) {
  GRID_STRIDE(idx, static_cast<long>(n) * n) {
    const long r = idx / n, c = idx % n;
    off[idx] = (r == c) ? make_double2(0.0, 0.0) : A[idx];
    if (r == c) diag[r] = A[idx];
  }
}

__global__ void precond_kernel(const double2 *R, const double2 *w, const double2 *d, int nr,
                               long dim, double2 *x) {
  GRID_STRIDE(idx, static_cast<long>(nr) * dim) {
    const long r = idx / dim, k = idx % dim;
    double2 den = csub(w[r], d[k]);
    const double m = hypot(den.x, den.y);
    if (m < 1e-8) den = make_double2(1e-8, 0.0);
    const double dd = den.x * den.x + den.y * den.y;
    x[idx] = cmul(R[idx], make_double2(den.x / dd, -den.y / dd));
  }
}

__global__ void scale_rows_kernel(double2 *x, const double2 *dots, int nr, long dim) {
  GRID_STRIDE(idx, static_cast<long>(nr) * dim) {
    const long r = idx / dim;
    const double nrm = sqrt(fmax(dots[r].x, 1e-300));
    x[idx] = cscale(1.0 / nrm, x[idx]);
  }
}

__global__ void add_diag_kernel(double2 *A, const double *diag, int n) {
  GRID_STRIDE(i, n) { A[i * static_cast<long>(n) + i].x += diag[i]; }
}

__device__ __forceinline__ double2 cmul_rn(double2 a, double2 b) {
  return make_double2(__dsub_rn(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)),
                      __dadd_rn(__dmul_rn(a.x, b.y), __dmul_rn(a.y, b.x)));
}

__global__ void dump_kernel(const double2 *Lpr, long aP, long ap, long ar, const double2 *Lqs,
                            long bP, long bq, long bs, const double2 *Lps, long cP, long cp,
                            long cs, const double2 *Lqr, long dP, long dq, long dr, int X, int np,
                            int nq, int nr, int ns, double2 *out) {
  const long total = static_cast<long>(np) * nq * nr * ns;
  GRID_STRIDE(idx, total) {
    const int s = static_cast<int>(idx % ns);
    const int r = static_cast<int>((idx / ns) % nr);
    const int q = static_cast<int>((idx / (static_cast<long>(ns) * nr)) % nq);
    const int p = static_cast<int>(idx / (static_cast<long>(ns) * nr * nq));
    double2 acc = make_double2(0.0, 0.0);
    for (int P = 0; P < X; ++P) {
      const double2 d1 = cmul_rn(Lpr[P * aP + p * ap + r * ar], Lqs[P * bP + q * bq + s * bs]);
      const double2 d2 = cmul_rn(Lps[P * cP + p * cp + s * cs], Lqr[P * dP + q * dq + r * dr]);
      const double2 t = make_double2(__dsub_rn(d1.x, d2.x), __dsub_rn(d1.y, d2.y));
      acc = make_double2(__dadd_rn(acc.x, t.x), __dadd_rn(acc.y, t.y));
    }
    out[idx] = acc;
  }
}

}  // namespace

// t[j'][a][b] = (G[j'][a][b] - G[j'][b][a]) / (eps_i + eps_j - eps_a - eps_b)
// for j = i + 1 + j' (MP2 amplitudes of the pairs (i, j > i), Eq. 24's t)
__global__ void mp2_pair_kernel(const double2 *G, const double *eps, int o, int v, int i, int nj,
                                double2 *t) {
  const long vv = static_cast<long>(v) * v;
  GRID_STRIDE(idx, static_cast<long>(nj) * vv) {
    const long jp = idx / vv, r = idx - jp * vv;
    const int a = static_cast<int>(r / v), b = static_cast<int>(r - (r / v) * v);
    const double2 g1 = G[idx], g2 = G[jp * vv + static_cast<long>(b) * v + a];
    const double D = eps[i] + eps[i + 1 + jp] - eps[o + a] - eps[o + b];
    t[idx] = make_double2((g1.x - g2.x) / D, (g1.y - g2.y) / D);
  }
}

void mp2_pair_amplitudes(const cplx *G, const double *eps, int o, int v, int i, int nj, cplx *t,
                         cudaStream_t st) {
  if (nj <= 0) return;
  mp2_pair_kernel<<<grid_for(static_cast<long>(nj) * v * v), 256, 0, st>>>(G, eps, o, v, i, nj, t);
  LAUNCH_CHECK();
  count_launch();
}

void split_cholesky(const cplx *chunk, int np, int p0, int o, int v, cplx *Loo, cplx *Lov,
                    cplx *Lvo, cplx *Lvv, unsigned long long *stats, cudaStream_t st) {
  const long total = static_cast<long>(np) * (o + v) * (o + v);
  split_kernel<<<grid_for(total), 256, 0, st>>>(chunk, np, p0, o, v, Loo, Lov, Lvo, Lvv, stats);
  LAUNCH_CHECK();
  count_launch();
}

inline dim3 grid2d(int o, int v) {
  const int vv = v * v;
  const unsigned gx = static_cast<unsigned>(std::min((vv + 255) / 256, 64));
  const unsigned gy = static_cast<unsigned>(std::min(o * o, 65535));
  return dim3(gx, gy);
}

namespace {
template <bool ANTI>
void t1t1_launch(const cplx *t1, const cplx *t2, cplx *out0, cplx *out1, int o, int v, double c0,
                 double f0, double f1, bool f32, cudaStream_t st, float *mx) {
  if (o <= 0 || v <= 0) return;
  if (static_cast<long>(o) * o > 65535) fail(CC_ERR_ARG, "t1t1: n_occ too large");
  const int c0_half = c0 == 1.0 ? 0 : (c0 == 0.5 ? 1 : -1);
  dim3 grid(static_cast<unsigned>((v + 31) / 32), static_cast<unsigned>(o * o));
  const size_t sm = 2 * static_cast<size_t>(v) * (f32 ? sizeof(float2) : sizeof(double2));
  if (sm > 48 * 1024) {
    CUDA_CHECK(cudaFuncSetAttribute(f32 ? t1t1_kernel<float2, ANTI> : t1t1_kernel<double2, ANTI>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(sm)));
  }
  if (mx) CUDA_CHECK(cudaMemsetAsync(mx, 0, 3 * sizeof(float), st));
  if (f32)
    t1t1_kernel<float2, ANTI><<<grid, 256, sm, st>>>(t1, t2, out0, out1, o, v, c0_half, c0,
                                                     static_cast<float>(f0), static_cast<float>(f1),
                                                     mx);
  else
    t1t1_kernel<double2, ANTI><<<grid, 256, sm, st>>>(t1, t2, out0, out1, o, v, c0_half, c0,
                                                      static_cast<float>(f0), static_cast<float>(f1),
                                                      mx);
  LAUNCH_CHECK();
  count_launch();
}
}  // namespace

void make_tau(const cplx *t1, const cplx *t2, cplx *out, int o, int v, double f, cudaStream_t st,
              bool fp32_t1, float *mx) {
  if (!fp32_t1 && f != 1.0 && f != 0.5) fail(CC_ERR_ARG, "make_tau: f must be 1 or 1/2");
  t1t1_launch<true>(t1, t2, out, nullptr, o, v, 1.0, f, 0.0, fp32_t1, st, mx);
}

void make_tau_pair(const cplx *t1, const cplx *t2, cplx *tau, cplx *taut, int o, int v,
                   cudaStream_t st, bool fp32_t1, float *mx) {
  t1t1_launch<true>(t1, t2, tau, taut, o, v, 1.0, 1.0, 0.5, fp32_t1, st, mx);
}

void jacobi(const cplx *R1, const cplx *R2, const double *eps, int o, int v, cplx *t1, cplx *t2,
            cudaStream_t st) {
  if (static_cast<long>(o) * v > static_cast<long>(v) * v)
    fail(CC_ERR_UNSUPPORTED, "jacobi: n_occ > n_virt is not supported");
  jacobi_kernel<<<grid2d(o, v), 256, 0, st>>>(R1, R2, eps, o, v, t1, t2);
  LAUNCH_CHECK();
  count_launch();
}

void mp2_amplitudes(const cplx *oovv, const double *eps, int o, int v, cplx *t1, cplx *t2,
                    cudaStream_t st) {
  mp2_kernel<<<grid_for(static_cast<long>(o) * o * v * v), 256, 0, st>>>(oovv, eps, o, v, t1, t2);
  LAUNCH_CHECK();
  count_launch();
}

void pack_amps(const cplx *t1, const cplx *t2, int o, int v, const int *ij_i, const int *ij_j,
               const int *ab_a, const int *ab_b, cplx *vec, cudaStream_t st) {
  const long n = static_cast<long>(o) * v +
                 static_cast<long>(o) * (o - 1) / 2 * (static_cast<long>(v) * (v - 1) / 2);
  pack_amps_kernel<<<grid_for(n), 256, 0, st>>>(t1, t2, o, v, ij_i, ij_j, ab_a, ab_b, vec);
  LAUNCH_CHECK();
  count_launch();
}

void unpack_amps(const cplx *vec, int o, int v, cplx *t1, cplx *t2, cudaStream_t st) {
  if (o <= 0 || v <= 0) return;
  if (static_cast<long>(o) * o > 65535) fail(CC_ERR_ARG, "unpack_amps: n_occ too large");
  dim3 grid(static_cast<unsigned>((v + 7) / 8), static_cast<unsigned>(o * o));
  unpack_amps_kernel<<<grid, 256, 0, st>>>(vec, o, v, t1, t2);
  LAUNCH_CHECK();
  count_launch();
}

void amp_denoms(const double *eps, int o, int v, const int *ij_i, const int *ij_j, const int *ab_a,
                const int *ab_b, double *inv, cudaStream_t st) {
  const long n = static_cast<long>(o) * v +
                 static_cast<long>(o) * (o - 1) / 2 * (static_cast<long>(v) * (v - 1) / 2);
  amp_denoms_kernel<<<grid_for(n), 256, 0, st>>>(eps, o, v, ij_i, ij_j, ab_a, ab_b, inv);
  LAUNCH_CHECK();
  count_launch();
}

namespace {
dim3 pair_grid(int o, int v) {
  const long nij = static_cast<long>(o) * (o - 1) / 2;
  const long nab = static_cast<long>(v) * (v - 1) / 2;
  if (nij > 65535) fail(CC_ERR_ARG, "packed amplitudes: n_occ too large");
  const long gx = std::max<long>(1, std::min<long>((nab + 255) / 256, std::max<long>(1, 4096 / std::max<long>(nij, 1))));
  return dim3(static_cast<unsigned>(gx), static_cast<unsigned>(std::max<long>(nij, 1)));
}
}  // namespace

void jacobi_packed(const cplx *R1, const cplx *R2, const double *inv, int o, int v, const int *ij_i,
                   const int *ij_j, const int *ab_a, const int *ab_b, cplx *vec, cudaStream_t st) {
  if (o <= 0 || v <= 0) return;
  jacobi_packed_kernel<<<pair_grid(o, v), 256, 0, st>>>(R1, R2, inv, o, v, ij_i, ij_j, ab_a, ab_b,
                                                       vec);
  LAUNCH_CHECK();
  count_launch();
}

long energy_scratch_len(int o, int v) {
  const dim3 g = pair_grid(o, v);
  return static_cast<long>(g.x) * g.y;
}

void energy_packed(const cplx *oovv, const cplx *vec, int o, int v, const int *ij_i,
                   const int *ij_j, const int *ab_a, const int *ab_b, bool f32, cplx *scratch,
                   long scratch_len, cplx *res, cudaStream_t st) {
  const long nij = static_cast<long>(o) * (o - 1) / 2;
  if (nij == 0 || v < 2) {
    CUDA_CHECK(cudaMemsetAsync(res, 0, sizeof(cplx), st));
    return;
  }
  dim3 grid = pair_grid(o, v);
  while (static_cast<long>(grid.x) * grid.y > scratch_len && grid.x > 1) grid.x = (grid.x + 1) / 2;
  if (static_cast<long>(grid.x) * grid.y > scratch_len) fail(CC_ERR_ARG, "energy: scratch too small");
  if (f32)
    energy_packed_kernel<true><<<grid, 256, 0, st>>>(oovv, vec, o, v, ij_i, ij_j, ab_a, ab_b, scratch);
  else
    energy_packed_kernel<false><<<grid, 256, 0, st>>>(oovv, vec, o, v, ij_i, ij_j, ab_a, ab_b, scratch);
  LAUNCH_CHECK();
  sum_partials_kernel<<<1, 256, 0, st>>>(scratch, static_cast<long>(grid.x) * grid.y, res);
  LAUNCH_CHECK();
  count_launch(2);
}

void diis_solve(const cplx *B, int m, int ldb, cplx *coef, int *status, cudaStream_t st) {
  if (m > 16) fail(CC_ERR_ARG, "diis_solve: at most 16 vectors");
  diis_solve_kernel<<<1, 32, 0, st>>>(B, m, ldb, coef, status);
  LAUNCH_CHECK();
  count_launch();
}

void diis_combine(cplx *const *vecs, const cplx *coef, int m, long n, cplx *out, cudaStream_t st) {
  VecPtrs vp;
  for (int i = 0; i < m; ++i) vp.p[i] = vecs[i];
  combine_kernel<<<grid_for(n), 256, 0, st>>>(vp, coef, m, n, out);
  LAUNCH_CHECK();
  count_launch();
}

void ladder_antisym(const void *V, bool f32, int v, int a0, int nA, long p0, long p1,
                    const int *pair_a, const int *pair_b, const int *cd_c, const int *cd_d,
                    int tier, void *hi, void *lo, long kp, cplx *w64, cudaStream_t st,
                    const float *amax) {
  (void)nA;
  const long ncd = static_cast<long>(v) * (v - 1) / 2;
  const long np = p1 - p0;
  if (np <= 0) return;
  if (tier == TIER_FP64) {
    antisym_kernel<2><<<grid_for(np * ncd), 256, 0, st>>>(V, f32, v, a0, p0, p1, pair_a, pair_b,
                                                         cd_c, cd_d, ncd, nullptr, nullptr, 0, w64);
    LAUNCH_CHECK();
    count_launch();
    return;
  }
  if (!f32) fail(CC_ERR_ARG, "ladder_antisym: tensor-core tiers take an FP32 slab");
  if (tier_scaled(tier) && !amax) fail(CC_ERR_ARG, "ladder_antisym: FP16 needs the W bound");
  const int nt = (v + 31) / 32;
  // one wave of resident blocks, each walking many (a, b) pairs: a grid
  // beyond what the SMs hold at once would leave a last, mostly empty wave
  const long ntp = static_cast<long>(nt) * (nt + 1) / 2;
  const int pt = tier == TIER_BF16X3 ? 1 : tier == TIER_FP16 ? 2 : tier == TIER_FP16X3 ? 3 : 0;
  static int resident[4] = {0, 0, 0, 0};
  if (!resident[pt]) {
    int dev = 0, sms = 0, per_sm = 0;
    CUDA_CHECK(cudaGetDevice(&dev));
    CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const void *k = pt == 1 ? reinterpret_cast<const void *>(antisym_tile_kernel<1>)
                    : pt == 2 ? reinterpret_cast<const void *>(antisym_tile_kernel<2>)
                    : pt == 3 ? reinterpret_cast<const void *>(antisym_tile_kernel<3>)
                              : reinterpret_cast<const void *>(antisym_tile_kernel<0>);
    CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, 0));
    resident[pt] = std::max(1, sms * per_sm);
  }
  dim3 grid(static_cast<unsigned>(ntp),
            static_cast<unsigned>(std::max<long>(1, std::min<long>(np, resident[pt] / ntp))));
  const float2 *Vf = reinterpret_cast<const float2 *>(V);
  if (tier == TIER_BF16X3) {
    antisym_tile_kernel<1><<<grid, dim3(32, 8), 0, st>>>(Vf, v, a0, p0, np, pair_a, pair_b, hi, lo,
                                                         kp, nt, nullptr);
  } else if (tier == TIER_FP16) {
    antisym_tile_kernel<2><<<grid, dim3(32, 8), 0, st>>>(Vf, v, a0, p0, np, pair_a, pair_b, hi,
                                                         nullptr, kp, nt, amax);
  } else if (tier == TIER_FP16X3) {
    antisym_tile_kernel<3><<<grid, dim3(32, 8), 0, st>>>(Vf, v, a0, p0, np, pair_a, pair_b, hi, lo,
                                                         kp, nt, amax);
  } else {
    antisym_tile_kernel<0><<<grid, dim3(32, 8), 0, st>>>(Vf, v, a0, p0, np, pair_a, pair_b, hi,
                                                         tier == TIER_TF32 ? nullptr : lo, kp, nt,
                                                         nullptr);
  }
  LAUNCH_CHECK();
  count_launch();
  if (kp > 2 * ncd) {
    const unsigned gt = grid_for(np * (kp - 2 * ncd));
    if (tier == TIER_TF32 || tier == TIER_TF32X3) {
      zero_tail<float><<<gt, 256, 0, st>>>(reinterpret_cast<float *>(hi), np, 2 * ncd, kp);
      if (tier == TIER_TF32X3)
        zero_tail<float><<<gt, 256, 0, st>>>(reinterpret_cast<float *>(lo), np, 2 * ncd, kp);
    } else if (tier == TIER_BF16X3) {
      zero_tail<__nv_bfloat16><<<gt, 256, 0, st>>>(reinterpret_cast<__nv_bfloat16 *>(hi), np,
                                                    2 * ncd, kp);
      zero_tail<__nv_bfloat16><<<gt, 256, 0, st>>>(reinterpret_cast<__nv_bfloat16 *>(lo), np,
                                                    2 * ncd, kp);
    } else {
      zero_tail<__half><<<gt, 256, 0, st>>>(reinterpret_cast<__half *>(hi), np, 2 * ncd, kp);
      if (tier == TIER_FP16X3)
        zero_tail<__half><<<gt, 256, 0, st>>>(reinterpret_cast<__half *>(lo), np, 2 * ncd, kp);
    }
    LAUNCH_CHECK();
    count_launch();
  }
}


void unpack_pairs_add(const cplx *R, int o, int v, const int *ij_i, const int *ij_j,
                      const int *ab_a, const int *ab_b, cplx *R2, cudaStream_t st) {
  const long n = static_cast<long>(o) * (o - 1) / 2 * (static_cast<long>(v) * (v - 1) / 2);
  if (n <= 0) return;
  const long nij = static_cast<long>(o) * (o - 1) / 2;
  const int nt = (v + 31) / 32;
  if (nij <= 65535) {
    dim3 grid(static_cast<unsigned>(static_cast<long>(nt) * (nt + 1) / 2), static_cast<unsigned>(nij));
    unpack_pairs_tile_kernel<<<grid, dim3(32, 8), 0, st>>>(R, o, v, ij_i, ij_j, R2, nt);
  } else {
    unpack_pairs_kernel<<<grid_for(n), 256, 0, st>>>(R, o, v, ij_i, ij_j, ab_a, ab_b, R2);
  }
  LAUNCH_CHECK();
  count_launch();
}

void make_pairs(int n, int *pi, int *pj, cudaStream_t st) {
  const long np = static_cast<long>(n) * (n - 1) / 2;
  if (np <= 0) return;
  pairs_kernel<<<grid_for(np), 256, 0, st>>>(n, pi, pj);
  LAUNCH_CHECK();
  count_launch();
}

void ip_unpack(const cplx *vec, int k, int o, int v, cplx *r1, cplx *r2, cudaStream_t st) {
  ip_unpack_kernel<<<grid_for(static_cast<long>(k) * o * o * v), 256, 0, st>>>(vec, k, o, v, r1, r2);
  LAUNCH_CHECK();
  count_launch();
}

void ip_pack(const cplx *r1, const cplx *r2, int k, int o, int v, cplx *vec, cudaStream_t st) {
  const long dim = o + static_cast<long>(o) * (o - 1) / 2 * v;
  ip_pack_kernel<<<grid_for(k * dim), 256, 0, st>>>(r1, r2, k, o, v, vec);
  LAUNCH_CHECK();
  count_launch();
}

void ip_diag(const cplx *Hoo, const cplx *Hvv, int o, int v, cplx *d, cudaStream_t st) {
  const long dim = o + static_cast<long>(o) * (o - 1) / 2 * v;
  ip_diag_kernel<<<grid_for(dim), 256, 0, st>>>(Hoo, Hvv, o, v, d);
  LAUNCH_CHECK();
  count_launch();
}

void ip_diag_apply(const cplx *r1, const cplx *r2, const cplx *doo, const cplx *dvv, int k, int o,
                   int v, cplx *s1, cplx *s2, cudaStream_t st) {
  ip_diag_apply_kernel<<<grid_for(static_cast<long>(k) * o * o * v), 256, 0, st>>>(r1, r2, doo, dvv, k,
                                                                                  o, v, s1, s2);
  LAUNCH_CHECK();
  count_launch();
}

void sigma_combine(cplx *s2, const cplx *tA, const cplx *tB, const cplx *tC, const cplx *X1,
                   const cplx *X2, int k, int o, int v, cudaStream_t st) {
  sigma_combine_kernel<<<grid_for(static_cast<long>(k) * o * o * v), 256, 0, st>>>(s2, tA, tB, tC, X1,
                                                                                  X2, k, o, v);
  LAUNCH_CHECK();
  count_launch();
}

void split_diag(const cplx *A, int n, cplx *off, cplx *diag, cudaStream_t st) {
  split_diag_kernel<<<grid_for(static_cast<long>(n) * n), 256, 0, st>>>(A, n, off, diag);
  LAUNCH_CHECK();
  count_launch();
}

void precondition(const cplx *R, const cplx *w, const cplx *d, int nr, long dim, cplx *x,
                  cudaStream_t st) {
  precond_kernel<<<grid_for(nr * dim), 256, 0, st>>>(R, w, d, nr, dim, x);
  LAUNCH_CHECK();
  count_launch();
}

void scale_rows_inv_sqrt(cplx *x, const cplx *dots, int nr, long dim, cudaStream_t st) {
  scale_rows_kernel<<<grid_for(nr * dim), 256, 0, st>>>(x, dots, nr, dim);
  LAUNCH_CHECK();
  count_launch();
}

void add_diag(cplx *A, const double *diag, int n, cudaStream_t st) {
  add_diag_kernel<<<grid_for(n), 256, 0, st>>>(A, diag, n);
  LAUNCH_CHECK();
  count_launch();
}

void dump_block(const cplx *Lpr, long aP, long ap, long ar, const cplx *Lqs, long bP, long bq,
                long bs, const cplx *Lps, long cP, long cp, long cs, const cplx *Lqr, long dP,
                long dq, long dr, int X, int np, int nq, int nr, int ns, cplx *out,
                cudaStream_t st) {
  const long total = static_cast<long>(np) * nq * nr * ns;
  dump_kernel<<<grid_for(total), 256, 0, st>>>(Lpr, aP, ap, ar, Lqs, bP, bq, bs, Lps, cP, cp, cs,
                                               Lqr, dP, dq, dr, X, np, nq, nr, ns, out);
  LAUNCH_CHECK();
  count_launch();
}

}  // namespace cdfns
