// Learned warm start: a per-element MLP that maps gauge-invariant features of
// a doubles element (i<j, a<b) to the complex ratio rho = t_CCSD / t_MP2, so
// that t0 = rho * t_MP2 starts CCSD closer to convergence. The plain MP2
// start stays the fallback, and the converged result does not depend on the
// start (the CCSD equations are the same).
//
// Network: 8 -> 64 -> 64 -> 2, ReLU, FP16 weights (an FP32 master copy is
// kept for Adam), FP32 accumulation. Forward, backward and Adam are the
// kernels below; the host drives training on contiguous minibatches of a
// caller-shuffled sample order.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "solver.h"

namespace cdfns {

namespace {

constexpr int F = 8, H = 64, O = 2;
constexpr int W1 = 0, B1 = W1 + H * F, W2 = B1 + H, B2 = W2 + H * H, W3 = B2 + H, B3 = W3 + O * H;
constexpr int NP = B3 + O;  // 4866 parameters

inline unsigned grid_for(long n, int threads = 256) {
  return static_cast<unsigned>(std::max<long>(1, std::min<long>((n + threads - 1) / threads, 152L * 32)));
}

// load FP16 weights into shared memory as floats
__device__ void load_params(const __half *w, float *s) {
  for (int k = threadIdx.x; k < NP; k += blockDim.x) s[k] = __half2float(w[k]);
  __syncthreads();
}

__device__ __forceinline__ void forward(const float *p, const float *x, float *h1, float *h2,
                                        float *y) {
#pragma unroll
  for (int u = 0; u < H; ++u) {
    float a = p[B1 + u];
#pragma unroll
    for (int f = 0; f < F; ++f) a = fmaf(p[W1 + u * F + f], x[f], a);
    h1[u] = fmaxf(a, 0.f);
  }
#pragma unroll
  for (int u = 0; u < H; ++u) {
    float a = p[B2 + u];
#pragma unroll
    for (int k = 0; k < H; ++k) a = fmaf(p[W2 + u * H + k], h1[k], a);
    h2[u] = fmaxf(a, 0.f);
  }
#pragma unroll
  for (int c = 0; c < O; ++c) {
    float a = p[B3 + c];
#pragma unroll
    for (int k = 0; k < H; ++k) a = fmaf(p[W3 + c * H + k], h2[k], a);
    y[c] = a;
  }
}

// Inference: rho = 1 + y (the network predicts the deviation from MP2).
__global__ void mlp_infer_kernel(const __half *w, const float *X, long n, float2 *rho) {
  __shared__ float p[NP];
  load_params(w, p);
  for (long s = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; s < n;
       s += static_cast<long>(gridDim.x) * blockDim.x) {
    float x[F], h1[H], h2[H], y[O];
#pragma unroll
    for (int f = 0; f < F; ++f) x[f] = X[s * F + f];
    forward(p, x, h1, h2, y);
    rho[s] = make_float2(1.f + y[0], y[1]);
  }
}

// Loss and gradient of L = sum_s w_s |y_s - target_s|^2 / n over samples
// [s0, s0 + n) of the order perm (or identity). Y holds (re, im, weight).
// Gradients accumulate in shared memory (atomics) and then in global FP32.
__global__ void mlp_grad_kernel(const __half *w, const float *X, const float *Y, const int *perm,
                                long s0, long n, float *grad, float *loss) {
  __shared__ float p[NP];
  __shared__ float g[NP];
  __shared__ float lsum;
  for (int k = threadIdx.x; k < NP; k += blockDim.x) g[k] = 0.f;
  if (threadIdx.x == 0) lsum = 0.f;
  load_params(w, p);
  const float inv_n = 1.f / static_cast<float>(n);
  for (long t = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; t < n;
       t += static_cast<long>(gridDim.x) * blockDim.x) {
    const long s = perm ? perm[s0 + t] : s0 + t;
    float x[F], h1[H], h2[H], y[O];
#pragma unroll
    for (int f = 0; f < F; ++f) x[f] = X[s * F + f];
    forward(p, x, h1, h2, y);
    const float wt = Y[s * 3 + 2];
    float dy[O];
    float l = 0.f;
#pragma unroll
    for (int c = 0; c < O; ++c) {
      const float e = y[c] - Y[s * 3 + c];
      l += wt * e * e;
      dy[c] = 2.f * wt * e * inv_n;
    }
    atomicAdd(&lsum, l * inv_n);
    // layer 3
    float dh2[H];
#pragma unroll 8
    for (int k = 0; k < H; ++k) {
      float a = 0.f;
#pragma unroll
      for (int c = 0; c < O; ++c) {
        atomicAdd(&g[W3 + c * H + k], dy[c] * h2[k]);
        a = fmaf(p[W3 + c * H + k], dy[c], a);
      }
      dh2[k] = h2[k] > 0.f ? a : 0.f;
    }
#pragma unroll
    for (int c = 0; c < O; ++c) atomicAdd(&g[B3 + c], dy[c]);
    // layer 2
    float dh1[H];
#pragma unroll 4
    for (int k = 0; k < H; ++k) dh1[k] = 0.f;
    for (int u = 0; u < H; ++u) {
      if (dh2[u] == 0.f) continue;
      atomicAdd(&g[B2 + u], dh2[u]);
#pragma unroll 8
      for (int k = 0; k < H; ++k) {
        atomicAdd(&g[W2 + u * H + k], dh2[u] * h1[k]);
        dh1[k] = fmaf(p[W2 + u * H + k], dh2[u], dh1[k]);
      }
    }
    // layer 1
    for (int u = 0; u < H; ++u) {
      if (h1[u] <= 0.f || dh1[u] == 0.f) continue;
      atomicAdd(&g[B1 + u], dh1[u]);
#pragma unroll
      for (int f = 0; f < F; ++f) atomicAdd(&g[W1 + u * F + f], dh1[u] * x[f]);
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < NP; k += blockDim.x) atomicAdd(&grad[k], g[k]);
  if (threadIdx.x == 0) atomicAdd(loss, lsum);
}

// Adam on the FP32 master copy; the FP16 copy used by the kernels follows.
__global__ void adam_kernel(float *master, __half *w16, const float *grad, float *m, float *v,
                            float lr, float b1, float b2, float eps, float c1, float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= NP) return;
  const float gk = grad[k];
  m[k] = b1 * m[k] + (1.f - b1) * gk;
  v[k] = b2 * v[k] + (1.f - b2) * gk * gk;
  const float mh = m[k] / c1, vh = v[k] / c2;
  master[k] -= lr * mh / (sqrtf(vh) + eps);
  w16[k] = __float2half_rn(master[k]);
}

__global__ void to_half_kernel(const float *a, __half *b, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) b[k] = __float2half_rn(a[k]);
}

// <ab||ab> = sum_P (L^P_aa L^P_bb - L^P_ab L^P_ba), real for Hermitian L^P
__global__ void vv_diag_kernel(const double2 *Lvv, int X, int v, double *out) {
  const long vv = static_cast<long>(v) * v;
  for (long e = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; e < vv;
       e += static_cast<long>(gridDim.x) * blockDim.x) {
    const int a = static_cast<int>(e / v), b = static_cast<int>(e % v);
    double s = 0.0;
    for (int P = 0; P < X; ++P) {
      const double2 *L = Lvv + P * vv;
      const double2 aa = L[static_cast<long>(a) * v + a], bb = L[static_cast<long>(b) * v + b];
      const double2 ab = L[static_cast<long>(a) * v + b], ba = L[static_cast<long>(b) * v + a];
      s += (aa.x * bb.x - aa.y * bb.y) - (ab.x * ba.x - ab.y * ba.y);
    }
    out[e] = s;
  }
}

struct FeatArgs {
  const double2 *oovv, *oooo, *ovvo, *t2;
  const double *eps, *dvv;
  const int *ij_i, *ij_j, *ab_a, *ab_b;
  int o, v;
  long nab, stride, n;
  double g_scale, d_scale;
};

// Features of sample s = unique element stride * s (packed (i<j, a<b) order):
// log10 |t_MP2|, D / d_scale, <ij||ij>, <ab||ab>, the sum and the spread of
// <ia||ia> + <jb||jb> and <ib||ib> + <ja||ja> (integrals / g_scale),
// (eps_i + eps_j) / d_scale, and |<ij||ab>| / g_scale. Every one is invariant
// under spinor phase changes and symmetric under i<->j, a<->b.
// Y (optional, needs converged t2): Re, Im of rho - 1 and the weight |t_MP2|^2.
__global__ void features_kernel(FeatArgs A, float *X, float *Y, double *wsum) {
  const int o = A.o, v = A.v;
  const long vv = static_cast<long>(v) * v, oo = static_cast<long>(o) * o;
  for (long s = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; s < A.n;
       s += static_cast<long>(gridDim.x) * blockDim.x) {
    const long q = s * A.stride;
    const long pij = q / A.nab, pab = q - (q / A.nab) * A.nab;
    const int i = A.ij_i[pij], j = A.ij_j[pij], a = A.ab_a[pab], b = A.ab_b[pab];
    const long e = ((static_cast<long>(i) * o + j) * v + a) * v + b;
    const double D = A.eps[i] + A.eps[j] - A.eps[o + a] - A.eps[o + b];
    const double2 g = A.oovv[e];
    // t_MP2 = conj(<ij||ab>) / D
    const double2 tm = make_double2(g.x / D, -g.y / D);
    const double at = sqrt(tm.x * tm.x + tm.y * tm.y);
    const double dij = A.oooo[((static_cast<long>(i) * o + j) * o + i) * o + j].x;
    const double dab = A.dvv[static_cast<long>(a) * v + b];
    // <ia||ia> = -<ia||ai> = -ovvo[i][a][a][i]
    auto dia = [&](int ii, int aa) {
      return -A.ovvo[((static_cast<long>(ii) * v + aa) * v + aa) * o + ii].x;
    };
    const double s1 = dia(i, a) + dia(j, b), s2 = dia(i, b) + dia(j, a);
    float *x = X + s * F;
    x[0] = static_cast<float>(log10(at + 1e-300));
    x[1] = static_cast<float>(D / A.d_scale);
    x[2] = static_cast<float>(dij / A.g_scale);
    x[3] = static_cast<float>(dab / A.g_scale);
    x[4] = static_cast<float>((s1 + s2) / A.g_scale);
    x[5] = static_cast<float>(fabs(s1 - s2) / A.g_scale);
    x[6] = static_cast<float>((A.eps[i] + A.eps[j]) / A.d_scale);
    x[7] = static_cast<float>(sqrt(g.x * g.x + g.y * g.y) / A.g_scale);
    if (Y) {
      const double2 tc = A.t2[e];
      const double den = tm.x * tm.x + tm.y * tm.y;
      // rho = tc / tm
      const double rr = (tc.x * tm.x + tc.y * tm.y) / den, ri = (tc.y * tm.x - tc.x * tm.y) / den;
      Y[s * 3 + 0] = static_cast<float>(rr - 1.0);
      Y[s * 3 + 1] = static_cast<float>(ri);
      Y[s * 3 + 2] = static_cast<float>(den);
      atomicAdd(wsum, den);
    }
  }
  (void)vv;
  (void)oo;
}

__global__ void scale_weights_kernel(float *Y, long n, const double *wsum) {
  const float inv = static_cast<float>(static_cast<double>(n) / *wsum);
  for (long s = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; s < n;
       s += static_cast<long>(gridDim.x) * blockDim.x)
    Y[s * 3 + 2] *= inv;
}

// packed t2 start: vec[n1 + q] = rho_q * t_MP2_q for every unique element
__global__ void apply_rho_kernel(FeatArgs A, const float2 *rho, double2 *vec, long n1) {
  const int o = A.o, v = A.v;
  for (long q = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; q < A.n;
       q += static_cast<long>(gridDim.x) * blockDim.x) {
    const long pij = q / A.nab, pab = q - (q / A.nab) * A.nab;
    const int i = A.ij_i[pij], j = A.ij_j[pij], a = A.ab_a[pab], b = A.ab_b[pab];
    const long e = ((static_cast<long>(i) * o + j) * v + a) * v + b;
    const double D = A.eps[i] + A.eps[j] - A.eps[o + a] - A.eps[o + b];
    const double2 g = A.oovv[e];
    const double2 tm = make_double2(g.x / D, -g.y / D);
    const double2 r = make_double2(rho[q].x, rho[q].y);
    vec[n1 + q] = cmul(r, tm);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
  }
}

// ---------------------------------------------------------------------------
// Learned Davidson start. A root seeded at the 1h element i starts from
// r_i = 1 and 2h1p elements rho_nu c_nu, with c_nu = M_nu,i / (d_i - d_nu)
// the first-order (Rayleigh-Schroedinger) component about the diagonal d of
// H-bar_IP, M_nu,i = -W_ibjk for nu = (j<k, b) the 2h1p <- 1h coupling, and
// rho_nu the same network's complex ratio (1 without a network). Training
// targets are the converged right vectors, scaled so that r_i = 1:
// rho_nu = r_nu / c_nu.
// ---------------------------------------------------------------------------
struct GuessArgs {
  const double2 *Hovoo, *oooo, *ovvo, *d, *R;
  const int *ij_i, *ij_j, *seed;
  int o, v, nroots;
  long n2, dim, stride, n;
  double g_scale, d_scale;
};

__device__ __forceinline__ double2 first_order_component(const GuessArgs &A, int i, long q,
                                                         double2 *num) {
  const int o = A.o, v = A.v;
  const long p = q / v;
  const int b = static_cast<int>(q - p * v);
  const int j = A.ij_i[p], k = A.ij_j[p];
  const double2 h = A.Hovoo[((static_cast<long>(i) * v + b) * o + j) * o + k];
  *num = make_double2(-h.x, -h.y);
  const double2 den = csub(A.d[i], A.d[o + q]);
  const double dd = den.x * den.x + den.y * den.y;
  if (!(dd > 0.0)) return make_double2(0.0, 0.0);
  // num / den
  return make_double2((num->x * den.x + num->y * den.y) / dd, (num->y * den.x - num->x * den.y) / dd);
}

// Features of sample s = (root r, 2h1p element q) at flat index stride * s
// over [nroots][n2]: log10 |c|, (d_i - d_nu) / d_scale, |W_ibjk| / g_scale,
// whether the seed hole is j or k, d_i / d_scale, <jk||jk> / g_scale, and the
// sum and spread of <jb||jb>, <kb||kb> (/ g_scale); all invariant under
// spinor phase changes. Y (needs R): Re, Im of rho - 1 and the weight |c|^2.
__global__ void guess_features_kernel(GuessArgs A, float *X, float *Y, double *wsum) {
  const int o = A.o, v = A.v;
  for (long s = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; s < A.n;
       s += static_cast<long>(gridDim.x) * blockDim.x) {
    const long flat = s * A.stride;
    const int r = static_cast<int>(flat / A.n2);
    const long q = flat - static_cast<long>(r) * A.n2;
    const int i = A.seed[r];
    if (i < 0) {  // root not seeded at a 1h element: no features
      for (int f = 0; f < F; ++f) X[s * F + f] = 0.f;
      if (Y) Y[s * 3] = Y[s * 3 + 1] = Y[s * 3 + 2] = 0.f;
      continue;
    }
    const long p = q / v;
    const int b = static_cast<int>(q - p * v);
    const int j = A.ij_i[p], k = A.ij_j[p];
    double2 num;
    const double2 c = first_order_component(A, i, q, &num);
    const double ac = sqrt(c.x * c.x + c.y * c.y);
    const double2 den = csub(A.d[i], A.d[o + q]);
    auto dia = [&](int ii, int aa) {  // <ia||ia> = -<ia||ai>
      return -A.ovvo[((static_cast<long>(ii) * v + aa) * v + aa) * o + ii].x;
    };
    const double djb = dia(j, b), dkb = dia(k, b);
    float *x = X + s * F;
    x[0] = static_cast<float>(log10(ac + 1e-30));
    x[1] = static_cast<float>(den.x / A.d_scale);
    x[2] = static_cast<float>(sqrt(num.x * num.x + num.y * num.y) / A.g_scale);
    x[3] = (i == j || i == k) ? 1.f : 0.f;
    x[4] = static_cast<float>(A.d[i].x / A.d_scale);
    x[5] = static_cast<float>(A.oooo[((static_cast<long>(j) * o + k) * o + j) * o + k].x / A.g_scale);
    x[6] = static_cast<float>((djb + dkb) / A.g_scale);
    x[7] = static_cast<float>(fabs(djb - dkb) / A.g_scale);
    if (Y) {
      const double2 *Rr = A.R + static_cast<long>(r) * A.dim;
      const double2 ri = Rr[i], rn = Rr[o + q];
      const double den_i = ri.x * ri.x + ri.y * ri.y;
      // t = r_nu / r_i, then rho = t / c
      const double tx = (rn.x * ri.x + rn.y * ri.y) / den_i, ty = (rn.y * ri.x - rn.x * ri.y) / den_i;
      const double cc = c.x * c.x + c.y * c.y;
      float *y = Y + s * 3;
      if (cc > 0.0) {
        y[0] = static_cast<float>((tx * c.x + ty * c.y) / cc - 1.0);
        y[1] = static_cast<float>((ty * c.x - tx * c.y) / cc);
        y[2] = static_cast<float>(cc);
        atomicAdd(wsum, cc);
      } else {
        y[0] = y[1] = y[2] = 0.f;
      }
    }
  }
}

// Starting vectors: V[r] = e_i + sum_nu rho_nu c_nu e_nu for the seeded roots
// (rho = 1 where no network is given), V zeroed beforehand by the caller.
__global__ void build_guess_kernel(GuessArgs A, const float2 *rho, double2 *V) {
  const int o = A.o;
  const long tot = static_cast<long>(A.nroots) * A.n2;
  for (long s = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; s < tot;
       s += static_cast<long>(gridDim.x) * blockDim.x) {
    const int r = static_cast<int>(s / A.n2);
    const long q = s - static_cast<long>(r) * A.n2;
    const int i = A.seed[r];
    if (i < 0) continue;
    double2 num;
    double2 c = first_order_component(A, i, q, &num);
    if (rho) c = cmul(make_double2(rho[s].x, rho[s].y), c);
    double2 *Vr = V + static_cast<long>(r) * A.dim;
    Vr[o + q] = c;
    if (q == 0) Vr[i] = make_double2(1.0, 0.0);
  }
}

}  // namespace

struct Mlp {
  Allocator al;
  cudaStream_t st = nullptr;
  Buf master, w16, m, v, grad, loss, ws;
  Buf X, Y;  // training set
  long n = 0, cap = 0;
  long step = 0;
  std::string last_error;
};

// Per-system feature inputs and scales; fills A (n = element count or
// sample count) and returns device buffers kept alive by the caller.
static void feature_setup(Ctx &c, FeatArgs &A, Buf &dvv_buf) {
  c.ensure_ready();
  c.ensure_pairs();
  const int o = c.o, v = c.v;
  dvv_buf.reset(&c.al, sizeof(double) * v * v);
  vv_diag_kernel<<<grid_for(static_cast<long>(v) * v), 256, 0, c.st>>>(c.Lvv.c(), c.X, v,
                                                                       dvv_buf.as<double>());
  LAUNCH_CHECK();
  count_launch();
  // scales from the small diagonal arrays (host)
  std::vector<cplx> oo(static_cast<size_t>(o) * o * o * o);
  CUDA_CHECK(cudaMemcpyAsync(oo.data(), c.oooo.p, sizeof(cplx) * oo.size(), cudaMemcpyDeviceToHost,
                             c.st));
  CUDA_CHECK(cudaStreamSynchronize(c.st));
  double g2 = 0;
  long cnt = 0;
  for (int i = 0; i < o; ++i)
    for (int j = i + 1; j < o; ++j) {
      const double d = oo[((static_cast<size_t>(i) * o + j) * o + i) * o + j].x;
      g2 += d * d;
      ++cnt;
    }
  double dm = 0;
  for (int i = 0; i < o; ++i) dm -= c.eps[i];
  for (int a = 0; a < v; ++a) dm += c.eps[o + a];
  A.oovv = c.oovv.c();
  A.oooo = c.oooo.c();
  A.ovvo = c.ovvo.c();
  A.t2 = c.t2.p ? c.t2.c() : nullptr;
  A.eps = c.eps_d.as<double>();
  A.dvv = dvv_buf.as<double>();
  A.ij_i = c.ij_i.as<int>();
  A.ij_j = c.ij_j.as<int>();
  A.ab_a = c.ab_a.as<int>();
  A.ab_b = c.ab_b.as<int>();
  A.o = o;
  A.v = v;
  A.nab = c.nab();
  A.g_scale = std::sqrt(g2 / std::max<long>(cnt, 1)) + 1e-300;
  A.d_scale = 2.0 * dm / (o + v);  // mean |eps|-weighted scale, of order one Eh
}

// Inputs of the Davidson-start kernels for a context with H-bar built: the
// IP diagonal d (device, filled here) and the same scales as the amplitude
// features.
static void guess_setup(Ctx &c, GuessArgs &A, Buf &dbuf, const int *seed_dev, int nroots) {
  if (!c.hbar_done) fail(CC_ERR_STATE, "the Davidson start needs H-bar (a converged ccsd_solve)");
  c.ensure_pairs();
  const int o = c.o, v = c.v;
  dbuf.reset(&c.al, sizeof(cplx) * c.dim_ip());
  ip_diag(c.Hoo.c(), c.Hvv.c(), o, v, dbuf.c(), c.st);
  FeatArgs F0;
  Buf dvv;
  feature_setup(c, F0, dvv);
  A.Hovoo = c.Hovoo.c();
  A.oooo = c.oooo.c();
  A.ovvo = c.ovvo.c();
  A.d = dbuf.c();
  A.R = nullptr;
  A.ij_i = c.ij_i.as<int>();
  A.ij_j = c.ij_j.as<int>();
  A.seed = seed_dev;
  A.o = o;
  A.v = v;
  A.nroots = nroots;
  A.n2 = c.nij() * v;
  A.dim = c.dim_ip();
  A.stride = 1;
  A.n = static_cast<long>(nroots) * A.n2;
  A.g_scale = F0.g_scale;
  A.d_scale = F0.d_scale;
}

void davidson_guess(Ctx &c, const std::vector<int> &seeds, cplx *V) {
  const int nr = static_cast<int>(seeds.size());
  Buf sd(&c.al, sizeof(int) * std::max(nr, 1));
  CUDA_CHECK(cudaMemcpyAsync(sd.p, seeds.data(), sizeof(int) * nr, cudaMemcpyHostToDevice, c.st));
  GuessArgs A;
  Buf dbuf;
  guess_setup(c, A, dbuf, sd.as<int>(), nr);
  CUDA_CHECK(cudaMemsetAsync(V, 0, sizeof(cplx) * nr * A.dim, c.st));
  Buf X, rho;
  const float2 *rp = nullptr;
  if (c.guess_mode == 2) {
    if (!c.guess_mlp) fail(CC_ERR_STATE, "learned Davidson start without a network");
    const Mlp *m = static_cast<const Mlp *>(c.guess_mlp);
    X.reset(&c.al, sizeof(float) * A.n * F);
    rho.reset(&c.al, sizeof(float2) * A.n);
    guess_features_kernel<<<grid_for(A.n), 256, 0, c.st>>>(A, X.as<float>(), nullptr, nullptr);
    LAUNCH_CHECK();
    mlp_infer_kernel<<<grid_for(A.n, 128), 128, 0, c.st>>>(m->w16.as<__half>(), X.as<float>(), A.n,
                                                          rho.as<float2>());
    LAUNCH_CHECK();
    count_launch(2);
    rp = rho.as<float2>();
  }
  build_guess_kernel<<<grid_for(A.n), 256, 0, c.st>>>(A, rp, V);
  LAUNCH_CHECK();
  count_launch();
  // roots not seeded at a 1h element start as unit vectors at their seed
  const cplx one = mk(1.0, 0.0);
  for (int r = 0; r < nr; ++r)
    if (seeds[r] < 0) {
      const long pos = -2 - seeds[r];  // encoded position of the 2h1p element
      CUDA_CHECK(cudaMemcpyAsync(V + static_cast<long>(r) * A.dim + pos, &one, sizeof(cplx),
                                 cudaMemcpyHostToDevice, c.st));
    }
  CUDA_CHECK(cudaStreamSynchronize(c.st));
}

}  // namespace cdfns

struct cc_mlp {
  cdfns::Mlp m;
};

using cdfns::Buf;
using cdfns::Mlp;

namespace {

template <class F>
int guard(cc_mlp *p, F &&f) {
  try {
    return f();
  } catch (const cdfns::Error &e) {
    if (p) p->m.last_error = e.msg;
    return e.code;
  } catch (const std::exception &e) {
    if (p) p->m.last_error = e.what();
    return CC_ERR_CUDA;
  }
}

}  // namespace

extern "C" {

int cc_mlp_num_params(void) { return cdfns::NP; }

int cc_mlp_create(cc_mlp **out) {
  if (!out) return CC_ERR_ARG;
  *out = nullptr;
  cc_mlp *p = new (std::nothrow) cc_mlp;
  if (!p) return CC_ERR_OOM;
  const int rc = guard(p, [&] {
    Mlp &m = p->m;
    const size_t nb = sizeof(float) * cdfns::NP;
    m.master.reset(&m.al, nb);
    m.w16.reset(&m.al, sizeof(__half) * cdfns::NP);
    m.m.reset(&m.al, nb);
    m.v.reset(&m.al, nb);
    m.grad.reset(&m.al, nb);
    m.loss.reset(&m.al, sizeof(float) * 4);
    m.ws.reset(&m.al, sizeof(double) * 4);
    CUDA_CHECK(cudaMemset(m.master.p, 0, nb));
    CUDA_CHECK(cudaMemset(m.w16.p, 0, sizeof(__half) * cdfns::NP));
    CUDA_CHECK(cudaMemset(m.m.p, 0, nb));
    CUDA_CHECK(cudaMemset(m.v.p, 0, nb));
    return CC_OK;
  });
  if (rc != CC_OK) {
    delete p;
    return rc;
  }
  *out = p;
  return CC_OK;
}

void cc_mlp_free(cc_mlp *p) { delete p; }

const char *cc_mlp_last_error(const cc_mlp *p) { return p ? p->m.last_error.c_str() : ""; }

int cc_mlp_set_params(cc_mlp *p, const float *host, int n) {
  if (!p || !host || n != cdfns::NP) return CC_ERR_ARG;
  return guard(p, [&] {
    Mlp &m = p->m;
    CUDA_CHECK(cudaMemcpy(m.master.p, host, sizeof(float) * n, cudaMemcpyHostToDevice));
    cdfns::to_half_kernel<<<(n + 255) / 256, 256, 0, m.st>>>(m.master.as<float>(), m.w16.as<__half>(), n);
    LAUNCH_CHECK();
    CUDA_CHECK(cudaMemsetAsync(m.m.p, 0, sizeof(float) * n, m.st));
    CUDA_CHECK(cudaMemsetAsync(m.v.p, 0, sizeof(float) * n, m.st));
    CUDA_CHECK(cudaStreamSynchronize(m.st));
    m.step = 0;
    return CC_OK;
  });
}

int cc_mlp_get_params(const cc_mlp *cp, float *host, int n) {
  cc_mlp *p = const_cast<cc_mlp *>(cp);
  if (!p || !host || n != cdfns::NP) return CC_ERR_ARG;
  return guard(p, [&] {
    CUDA_CHECK(cudaMemcpy(host, p->m.master.p, sizeof(float) * n, cudaMemcpyDeviceToHost));
    return CC_OK;
  });
}

int cc_mlp_add_samples(cc_mlp *p, cc_ctx *ctx, long max_samples) {
  if (!p || !ctx || max_samples < 1) return CC_ERR_ARG;
  return guard(p, [&] {
    cdfns::Ctx &c = ctx->c;
    if (!c.ccsd_done) cdfns::fail(CC_ERR_STATE, "add_samples needs converged CCSD amplitudes");
    Mlp &m = p->m;
    cdfns::FeatArgs A;
    Buf dvv;
    cdfns::feature_setup(c, A, dvv);
    const long total = c.nij() * c.nab();
    A.stride = std::max<long>(1, total / max_samples);
    A.n = total / A.stride;
    if (m.n + A.n > m.cap) {
      const long cap = (m.n + A.n) * 2;
      Buf X2(&m.al, sizeof(float) * cap * cdfns::F), Y2(&m.al, sizeof(float) * cap * 3);
      if (m.n) {
        CUDA_CHECK(cudaMemcpy(X2.p, m.X.p, sizeof(float) * m.n * cdfns::F, cudaMemcpyDeviceToDevice));
        CUDA_CHECK(cudaMemcpy(Y2.p, m.Y.p, sizeof(float) * m.n * 3, cudaMemcpyDeviceToDevice));
      }
      m.X = std::move(X2);
      m.Y = std::move(Y2);
      m.cap = cap;
    }
    CUDA_CHECK(cudaMemsetAsync(m.ws.p, 0, sizeof(double), c.st));
    float *Xp = m.X.as<float>() + m.n * cdfns::F, *Yp = m.Y.as<float>() + m.n * 3;
    cdfns::features_kernel<<<cdfns::grid_for(A.n), 256, 0, c.st>>>(A, Xp, Yp, m.ws.as<double>());
    LAUNCH_CHECK();
    cdfns::scale_weights_kernel<<<cdfns::grid_for(A.n), 256, 0, c.st>>>(Yp, A.n, m.ws.as<double>());
    LAUNCH_CHECK();
    cdfns::count_launch(2);
    CUDA_CHECK(cudaStreamSynchronize(c.st));
    m.n += A.n;
    return CC_OK;
  });
}

int cc_mlp_num_samples(const cc_mlp *p, long *n) {
  if (!p || !n) return CC_ERR_ARG;
  *n = p->m.n;
  return CC_OK;
}

// Loss and gradient for samples [s0, s0 + n) of the training set taken in the
// order perm_dev (device int array over the set, or NULL for identity).
static void grad_batch(Mlp &m, const int *perm, long s0, long n, const float *X, const float *Y) {
  CUDA_CHECK(cudaMemsetAsync(m.grad.p, 0, sizeof(float) * cdfns::NP, m.st));
  CUDA_CHECK(cudaMemsetAsync(m.loss.p, 0, sizeof(float), m.st));
  const unsigned blocks = static_cast<unsigned>(std::min<long>((n + 127) / 128, 64));
  cdfns::mlp_grad_kernel<<<blocks, 128, 0, m.st>>>(m.w16.as<__half>(), X, Y, perm, s0, n,
                                                   m.grad.as<float>(), m.loss.as<float>());
  LAUNCH_CHECK();
  cdfns::count_launch();
}

int cc_mlp_train(cc_mlp *p, int steps, int batch, float lr, const int *perm_host, long perm_len,
                 double *final_loss) {
  if (!p || steps < 0 || batch < 1 || !(lr > 0)) return CC_ERR_ARG;
  return guard(p, [&] {
    Mlp &m = p->m;
    if (m.n < batch) cdfns::fail(CC_ERR_STATE, "training set smaller than one batch");
    const long np = perm_host ? perm_len : m.n;
    if (perm_host && perm_len < batch) cdfns::fail(CC_ERR_ARG, "perm shorter than a batch");
    Buf perm(&m.al, sizeof(int) * std::max<long>(np, 1));
    if (perm_host) {
      for (long k = 0; k < perm_len; ++k)
        if (perm_host[k] < 0 || perm_host[k] >= m.n) cdfns::fail(CC_ERR_ARG, "perm index out of range");
      CUDA_CHECK(cudaMemcpy(perm.p, perm_host, sizeof(int) * perm_len, cudaMemcpyHostToDevice));
    }
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    float lh = 0.f;
    long pos = 0;
    for (int it = 0; it < steps; ++it) {
      if (pos + batch > np) pos = 0;
      grad_batch(m, perm_host ? perm.as<int>() : nullptr, pos, batch, m.X.as<float>(), m.Y.as<float>());
      pos += batch;
      ++m.step;
      const float c1 = 1.f - std::pow(b1, static_cast<float>(m.step));
      const float c2 = 1.f - std::pow(b2, static_cast<float>(m.step));
      cdfns::adam_kernel<<<(cdfns::NP + 255) / 256, 256, 0, m.st>>>(
          m.master.as<float>(), m.w16.as<__half>(), m.grad.as<float>(), m.m.as<float>(),
          m.v.as<float>(), lr, b1, b2, eps, c1, c2);
      LAUNCH_CHECK();
      cdfns::count_launch();
    }
    CUDA_CHECK(cudaMemcpyAsync(&lh, m.loss.p, sizeof(float), cudaMemcpyDeviceToHost, m.st));
    CUDA_CHECK(cudaStreamSynchronize(m.st));
    if (final_loss) *final_loss = lh;
    return CC_OK;
  });
}

int cc_mlp_loss_grad(cc_mlp *p, long n, const float *X_host, const float *Y_host, double *loss,
                     float *grad_host) {
  if (!p || n < 1 || !X_host || !Y_host || !loss || !grad_host) return CC_ERR_ARG;
  return guard(p, [&] {
    Mlp &m = p->m;
    Buf X(&m.al, sizeof(float) * n * cdfns::F), Y(&m.al, sizeof(float) * n * 3);
    CUDA_CHECK(cudaMemcpy(X.p, X_host, sizeof(float) * n * cdfns::F, cudaMemcpyHostToDevice));
    CUDA_CHECK(cudaMemcpy(Y.p, Y_host, sizeof(float) * n * 3, cudaMemcpyHostToDevice));
    grad_batch(m, nullptr, 0, n, X.as<float>(), Y.as<float>());
    float l = 0.f;
    CUDA_CHECK(cudaMemcpyAsync(&l, m.loss.p, sizeof(float), cudaMemcpyDeviceToHost, m.st));
    CUDA_CHECK(cudaMemcpyAsync(grad_host, m.grad.p, sizeof(float) * cdfns::NP, cudaMemcpyDeviceToHost,
                               m.st));
    CUDA_CHECK(cudaStreamSynchronize(m.st));
    *loss = l;
    return CC_OK;
  });
}

int cc_mlp_features(cc_ctx *ctx, long n, float *X_host) {
  if (!ctx || n < 1 || !X_host) return CC_ERR_ARG;
  cdfns::Ctx &c = ctx->c;
  try {
    cdfns::FeatArgs A;
    Buf dvv;
    cdfns::feature_setup(c, A, dvv);
    A.t2 = nullptr;
    A.stride = 1;
    A.n = std::min<long>(n, c.nij() * c.nab());
    Buf X(&c.al, sizeof(float) * A.n * cdfns::F);
    cdfns::features_kernel<<<cdfns::grid_for(A.n), 256, 0, c.st>>>(A, X.as<float>(), nullptr, nullptr);
    LAUNCH_CHECK();
    CUDA_CHECK(cudaMemcpyAsync(X_host, X.p, sizeof(float) * A.n * cdfns::F, cudaMemcpyDeviceToHost, c.st));
    CUDA_CHECK(cudaStreamSynchronize(c.st));
    return CC_OK;
  } catch (const cdfns::Error &e) {
    c.last_error = e.msg;
    return e.code;
  }
}

int cc_set_davidson_guess(cc_ctx *ctx, int mode, const cc_mlp *mlp) {
  if (!ctx || mode < 0 || mode > 2 || (mode == 2 && !mlp)) return CC_ERR_ARG;
  ctx->c.guess_mode = mode;
  ctx->c.guess_mlp = mode == 2 ? static_cast<const void *>(&mlp->m) : nullptr;
  return CC_OK;
}

int ipeom_guess_dev(cc_ctx *ctx, int n_roots, double *out_dev) {
  if (!ctx || n_roots < 1 || !out_dev) return CC_ERR_ARG;
  cdfns::Ctx &c = ctx->c;
  try {
    if (!c.ccsd_done) cdfns::fail(CC_ERR_STATE, "the Davidson start needs a converged ccsd_solve");
    if (!c.hbar_done) c.build_hbar();
    if (n_roots > c.dim_ip()) cdfns::fail(CC_ERR_ARG, "n_roots out of range");
    const long dim = c.dim_ip();
    Buf d(&c.al, sizeof(cdfns::cplx) * dim);
    cdfns::ip_diag(c.Hoo.c(), c.Hvv.c(), c.o, c.v, d.c(), c.st);
    std::vector<cdfns::cplx> dh(dim);
    CUDA_CHECK(cudaMemcpyAsync(dh.data(), d.p, sizeof(cdfns::cplx) * dim, cudaMemcpyDeviceToHost, c.st));
    CUDA_CHECK(cudaStreamSynchronize(c.st));
    std::vector<long> idx(dim);
    for (long k = 0; k < dim; ++k) idx[k] = k;
    std::stable_sort(idx.begin(), idx.end(), [&](long a, long b) { return dh[a].x < dh[b].x; });
    std::vector<int> seeds(n_roots);
    for (int r = 0; r < n_roots; ++r)
      seeds[r] = idx[r] < c.o ? static_cast<int>(idx[r]) : static_cast<int>(-2 - idx[r]);
    cdfns::cplx *V = reinterpret_cast<cdfns::cplx *>(out_dev);
    if (c.guess_mode == 0) {
      CUDA_CHECK(cudaMemsetAsync(V, 0, sizeof(cdfns::cplx) * n_roots * dim, c.st));
      const cdfns::cplx one = cdfns::mk(1.0, 0.0);
      for (int r = 0; r < n_roots; ++r)
        CUDA_CHECK(cudaMemcpyAsync(V + r * dim + idx[r], &one, sizeof(one), cudaMemcpyHostToDevice, c.st));
      CUDA_CHECK(cudaStreamSynchronize(c.st));
    } else {
      cdfns::davidson_guess(c, seeds, V);
    }
    return CC_OK;
  } catch (const cdfns::Error &e) {
    c.last_error = e.msg;
    return e.code;
  }
}

int cc_mlp_guess_features(cc_ctx *ctx, int seed, long n, float *X_host) {
  if (!ctx || seed < 0 || n < 1 || !X_host) return CC_ERR_ARG;
  cdfns::Ctx &c = ctx->c;
  try {
    if (seed >= c.o) cdfns::fail(CC_ERR_ARG, "seed must be a 1h element");
    Buf sd(&c.al, sizeof(int));
    CUDA_CHECK(cudaMemcpyAsync(sd.p, &seed, sizeof(int), cudaMemcpyHostToDevice, c.st));
    cdfns::GuessArgs A;
    Buf dbuf;
    cdfns::guess_setup(c, A, dbuf, sd.as<int>(), 1);
    A.n = std::min<long>(n, A.n2);
    Buf X(&c.al, sizeof(float) * A.n * cdfns::F);
    cdfns::guess_features_kernel<<<cdfns::grid_for(A.n), 256, 0, c.st>>>(A, X.as<float>(), nullptr,
                                                                        nullptr);
    LAUNCH_CHECK();
    CUDA_CHECK(cudaMemcpyAsync(X_host, X.p, sizeof(float) * A.n * cdfns::F, cudaMemcpyDeviceToHost, c.st));
    CUDA_CHECK(cudaStreamSynchronize(c.st));
    return CC_OK;
  } catch (const cdfns::Error &e) {
    c.last_error = e.msg;
    return e.code;
  }
}

int cc_mlp_add_guess_samples(cc_mlp *p, cc_ctx *ctx, long max_samples) {
  if (!p || !ctx || max_samples < 1) return CC_ERR_ARG;
  return guard(p, [&] {
    cdfns::Ctx &c = ctx->c;
    if (c.last_nr < 1) cdfns::fail(CC_ERR_STATE, "add_guess_samples needs a converged ipeom_solve");
    Mlp &m = p->m;
    const int nr = c.last_nr, o = c.o;
    const long dim = c.dim_ip();
    // seed of each converged root: its largest 1h element, for roots whose
    // 1h weight is at least one half (the others give no samples)
    std::vector<cdfns::cplx> R1(static_cast<size_t>(nr) * dim);
    CUDA_CHECK(cudaMemcpyAsync(R1.data(), c.last_R.p, sizeof(cdfns::cplx) * nr * dim,
                               cudaMemcpyDeviceToHost, c.st));
    CUDA_CHECK(cudaStreamSynchronize(c.st));
    std::vector<int> seeds(nr, -1);
    for (int r = 0; r < nr; ++r) {
      double w1 = 0, wt = 0, best = -1;
      for (long k = 0; k < dim; ++k) {
        const cdfns::cplx x = R1[static_cast<size_t>(r) * dim + k];
        const double a2 = x.x * x.x + x.y * x.y;
        wt += a2;
        if (k < o) {
          w1 += a2;
          if (a2 > best) {
            best = a2;
            seeds[r] = static_cast<int>(k);
          }
        }
      }
      if (w1 < 0.5 * wt) seeds[r] = -1;
    }
    Buf sd(&c.al, sizeof(int) * nr);
    CUDA_CHECK(cudaMemcpyAsync(sd.p, seeds.data(), sizeof(int) * nr, cudaMemcpyHostToDevice, c.st));
    cdfns::GuessArgs A;
    Buf dbuf;
    cdfns::guess_setup(c, A, dbuf, sd.as<int>(), nr);
    A.R = c.last_R.c();
    const long total = static_cast<long>(nr) * A.n2;
    A.stride = std::max<long>(1, total / max_samples);
    A.n = total / A.stride;
    if (m.n + A.n > m.cap) {
      const long cap = (m.n + A.n) * 2;
      Buf X2(&m.al, sizeof(float) * cap * cdfns::F), Y2(&m.al, sizeof(float) * cap * 3);
      if (m.n) {
        CUDA_CHECK(cudaMemcpy(X2.p, m.X.p, sizeof(float) * m.n * cdfns::F, cudaMemcpyDeviceToDevice));
        CUDA_CHECK(cudaMemcpy(Y2.p, m.Y.p, sizeof(float) * m.n * 3, cudaMemcpyDeviceToDevice));
      }
      m.X = std::move(X2);
      m.Y = std::move(Y2);
      m.cap = cap;
    }
    CUDA_CHECK(cudaMemsetAsync(m.ws.p, 0, sizeof(double), c.st));
    float *Xp = m.X.as<float>() + m.n * cdfns::F, *Yp = m.Y.as<float>() + m.n * 3;
    cdfns::guess_features_kernel<<<cdfns::grid_for(A.n), 256, 0, c.st>>>(A, Xp, Yp, m.ws.as<double>());
    LAUNCH_CHECK();
    cdfns::scale_weights_kernel<<<cdfns::grid_for(A.n), 256, 0, c.st>>>(Yp, A.n, m.ws.as<double>());
    LAUNCH_CHECK();
    cdfns::count_launch(2);
    CUDA_CHECK(cudaStreamSynchronize(c.st));
    m.n += A.n;
    return CC_OK;
  });
}

int cc_mlp_warm_start(cc_mlp *p, cc_ctx *ctx) {
  if (!p || !ctx) return CC_ERR_ARG;
  cdfns::Ctx &c = ctx->c;
  return guard(p, [&] {
    if (c.ccsd_done || c.amps_user) cdfns::fail(CC_ERR_STATE, "warm start must precede ccsd_solve");
    cdfns::FeatArgs A;
    Buf dvv;
    cdfns::feature_setup(c, A, dvv);
    A.t2 = nullptr;
    A.stride = 1;
    A.n = c.nij() * c.nab();
    const long n1 = static_cast<long>(c.o) * c.v;
    Buf X(&c.al, sizeof(float) * A.n * cdfns::F), rho(&c.al, sizeof(float2) * A.n);
    Buf vec(&c.al, sizeof(cdfns::cplx) * (n1 + A.n));
    cdfns::features_kernel<<<cdfns::grid_for(A.n), 256, 0, c.st>>>(A, X.as<float>(), nullptr, nullptr);
    LAUNCH_CHECK();
    cdfns::mlp_infer_kernel<<<cdfns::grid_for(A.n, 128), 128, 0, c.st>>>(
        p->m.w16.as<__half>(), X.as<float>(), A.n, rho.as<float2>());
    LAUNCH_CHECK();
    CUDA_CHECK(cudaMemsetAsync(vec.p, 0, sizeof(cdfns::cplx) * n1, c.st));
    cdfns::apply_rho_kernel<<<cdfns::grid_for(A.n), 256, 0, c.st>>>(A, rho.as<float2>(), vec.c(), n1);
    LAUNCH_CHECK();
    cdfns::count_launch(3);
    c.B(c.t1, n1);
    c.B(c.t2, static_cast<long>(c.o) * c.o * c.v * c.v);
    cdfns::unpack_amps(vec.c(), c.o, c.v, c.t1.c(), c.t2.c(), c.st);
    CUDA_CHECK(cudaStreamSynchronize(c.st));
    c.amps = true;
    c.hbar_done = false;
    return CC_OK;
  });
}

}  // extern "C"
