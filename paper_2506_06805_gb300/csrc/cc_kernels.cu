#include <cuda_bf16.h>

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
    if (p < o && q < o) Loo[(PP * o + p) * o + q] = x;
    else if (p < o) Lov[(PP * o + p) * v + (q - o)] = x;
    else if (q < o) Lvo[(PP * v + (p - o)) * o + q] = x;
    else Lvv[(PP * v + (p - o)) * v + (q - o)] = x;
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
__global__ void tau_kernel(const double2 *t1, const double2 *t2, double2 *out, int o, int v,
                           double f) {
  const int vv = v * v;
  for (int ij = blockIdx.y; ij < o * o; ij += gridDim.y) {
    const int i = ij / o, j = ij - (ij / o) * o;
    const long base = static_cast<long>(ij) * vv;
    for (int ab = blockIdx.x * blockDim.x + threadIdx.x; ab < vv; ab += gridDim.x * blockDim.x) {
      const int a = ab / v, b = ab - (ab / v) * v;
      const double2 x = csub(cmul(t1[i * v + a], t1[j * v + b]), cmul(t1[i * v + b], t1[j * v + a]));
      out[base + ab] = cadd(t2[base + ab], cscale(f, x));
    }
  }
}

// Same with the t1 t1 part formed in FP32 (for the tensor-core tiers, whose
// GEMMs round these operands to TF32/BF16 anyway; GB300's FP64 rate is low).
__global__ void tau32_kernel(const double2 *t1, const double2 *t2, double2 *out, int o, int v,
                             float f) {
  const int vv = v * v;
  for (int ij = blockIdx.y; ij < o * o; ij += gridDim.y) {
    const int i = ij / o, j = ij - (ij / o) * o;
    const long base = static_cast<long>(ij) * vv;
    for (int ab = blockIdx.x * blockDim.x + threadIdx.x; ab < vv; ab += gridDim.x * blockDim.x) {
      const int a = ab / v, b = ab - (ab / v) * v;
      const double2 p = t1[i * v + a], q = t1[j * v + b], r = t1[i * v + b], s = t1[j * v + a];
      const float2 pf = make_float2(static_cast<float>(p.x), static_cast<float>(p.y));
      const float2 qf = make_float2(static_cast<float>(q.x), static_cast<float>(q.y));
      const float2 rf = make_float2(static_cast<float>(r.x), static_cast<float>(r.y));
      const float2 sf = make_float2(static_cast<float>(s.x), static_cast<float>(s.y));
      const float xr = (pf.x * qf.x - pf.y * qf.y) - (rf.x * sf.x - rf.y * sf.y);
      const float xi = (pf.x * qf.y + pf.y * qf.x) - (rf.x * sf.y + rf.y * sf.x);
      const double2 t = t2[base + ab];
      out[base + ab] = make_double2(t.x + static_cast<double>(f * xr), t.y + static_cast<double>(f * xi));
    }
  }
}

__global__ void z_kernel(const double2 *t1, const double2 *t2, double2 *out, int o, int v,
                         double c2) {
  // out[j][n][f][b] = c2 t2[j][n][f][b] + t1[j][f] t1[n][b]
  const int vv = v * v;
  for (int jn = blockIdx.y; jn < o * o; jn += gridDim.y) {
    const int j = jn / o, n = jn - (jn / o) * o;
    const long base = static_cast<long>(jn) * vv;
    for (int fb = blockIdx.x * blockDim.x + threadIdx.x; fb < vv; fb += gridDim.x * blockDim.x) {
      const int f = fb / v, b = fb - (fb / v) * v;
      out[base + fb] = cadd(cscale(c2, t2[base + fb]), cmul(t1[j * v + f], t1[n * v + b]));
    }
  }
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

__global__ void unpack_amps_kernel(const double2 *vec, int o, int v, double2 *t1, double2 *t2) {
  const long n1 = static_cast<long>(o) * v;
  const long nab = static_cast<long>(v) * (v - 1) / 2;
  const long total = static_cast<long>(o) * o * v * v;
  GRID_STRIDE(idx, total) {
    const int b = static_cast<int>(idx % v);
    const int a = static_cast<int>((idx / v) % v);
    const int j = static_cast<int>((idx / (static_cast<long>(v) * v)) % o);
    const int i = static_cast<int>(idx / (static_cast<long>(v) * v * o));
    double2 x = make_double2(0.0, 0.0);
    if (i != j && a != b) {
      const int ii = min(i, j), jj = max(i, j), aa = min(a, b), bb = max(a, b);
      const double s = ((i < j) == (a < b)) ? 1.0 : -1.0;
      x = cscale(s, vec[n1 + pair_index(ii, jj, o) * nab + pair_index(aa, bb, v)]);
    }
    t2[idx] = x;
    if (idx < n1) t1[idx] = vec[idx];
  }
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

void make_tau(const cplx *t1, const cplx *t2, cplx *out, int o, int v, double f, cudaStream_t st,
              bool fp32_t1) {
  if (fp32_t1)
    tau32_kernel<<<grid2d(o, v), 256, 0, st>>>(t1, t2, out, o, v, static_cast<float>(f));
  else
    tau_kernel<<<grid2d(o, v), 256, 0, st>>>(t1, t2, out, o, v, f);
  LAUNCH_CHECK();
  count_launch();
}

void make_z(const cplx *t1, const cplx *t2, cplx *out, int o, int v, double c2, cudaStream_t st) {
  z_kernel<<<grid2d(o, v), 256, 0, st>>>(t1, t2, out, o, v, c2);
  LAUNCH_CHECK();
  count_launch();
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
  unpack_amps_kernel<<<grid_for(static_cast<long>(o) * o * v * v), 256, 0, st>>>(vec, o, v, t1, t2);
  LAUNCH_CHECK();
  count_launch();
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
                    int tier, void *hi, void *lo, long kp, cplx *w64, cudaStream_t st) {
  (void)nA;
  const long ncd = static_cast<long>(v) * (v - 1) / 2;
  const long np = p1 - p0;
  if (np <= 0) return;
  const unsigned g = grid_for(np * ncd);
  if (tier == TIER_FP64) {
    antisym_kernel<2><<<g, 256, 0, st>>>(V, f32, v, a0, p0, p1, pair_a, pair_b, cd_c, cd_d, ncd,
                                         nullptr, nullptr, 0, w64);
  } else if (tier == TIER_BF16X3) {
    antisym_kernel<1><<<g, 256, 0, st>>>(V, f32, v, a0, p0, p1, pair_a, pair_b, cd_c, cd_d, ncd, hi,
                                         lo, kp, nullptr);
    if (kp > 2 * ncd) {
      zero_tail<__nv_bfloat16><<<grid_for(np * (kp - 2 * ncd)), 256, 0, st>>>(
          reinterpret_cast<__nv_bfloat16 *>(hi), np, 2 * ncd, kp);
      zero_tail<__nv_bfloat16><<<grid_for(np * (kp - 2 * ncd)), 256, 0, st>>>(
          reinterpret_cast<__nv_bfloat16 *>(lo), np, 2 * ncd, kp);
      count_launch(2);
    }
  } else {
    antisym_kernel<0><<<g, 256, 0, st>>>(V, f32, v, a0, p0, p1, pair_a, pair_b, cd_c, cd_d, ncd, hi,
                                         tier == TIER_TF32 ? nullptr : lo, kp, nullptr);
    if (kp > 2 * ncd) {
      zero_tail<float><<<grid_for(np * (kp - 2 * ncd)), 256, 0, st>>>(reinterpret_cast<float *>(hi),
                                                                        np, 2 * ncd, kp);
      count_launch();
      if (tier != TIER_TF32) {
        zero_tail<float><<<grid_for(np * (kp - 2 * ncd)), 256, 0, st>>>(
            reinterpret_cast<float *>(lo), np, 2 * ncd, kp);
        count_launch();
      }
    }
  }
  LAUNCH_CHECK();
  count_launch();
}

void unpack_pairs_add(const cplx *R, int o, int v, const int *ij_i, const int *ij_j,
                      const int *ab_a, const int *ab_b, cplx *R2, cudaStream_t st) {
  const long n = static_cast<long>(o) * (o - 1) / 2 * (static_cast<long>(v) * (v - 1) / 2);
  if (n <= 0) return;
  unpack_pairs_kernel<<<grid_for(n), 256, 0, st>>>(R, o, v, ij_i, ij_j, ab_a, ab_b, R2);
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
