// Skinny complex products on the CUDA cores in FP32 (tensor-core tiers).
//
// Contractions over a short index (K <= 48: an occupied index, o) with one
// short free side (a t1 or Fock-like block) and one long side (a doubles-
// sized tensor) move far more bytes than they compute: on the tensor-core
// path they would pay for expanded operand planes and for 128-row tiles
// that are mostly padding. Here each thread owns one row of the long
// operand, keeps its K elements in registers, and sweeps the short operand,
// which sits in shared memory; consecutive threads take consecutive long
// rows, whose outputs are adjacent in memory for every use in this library.
// Products and sums are FP32 (24-bit mantissa, finer than TF32); the
// epilogue adds into the FP64 output.
#include "kernels.h"

namespace cdfns {

namespace {

constexpr int SK_THREADS = 256;
constexpr int SK_SMEM = 96 * 1024;

// beta_mode: 0 C = alpha P, 1 C += alpha P, 2 C = alpha P + beta C (FP64).
__device__ __forceinline__ double2 epilogue(float pr, float pi, double2 old, float2 al,
                                            int beta_mode, double2 beta) {
  const double xr = f32_to_f64(al.x * pr - al.y * pi);
  const double xi = f32_to_f64(al.x * pi + al.y * pr);
  if (beta_mode == 0) return make_double2(xr, xi);
  if (beta_mode == 1) return make_double2(old.x + xr, old.y + xi);
  return make_double2(beta.x * old.x - beta.y * old.y + xr, beta.x * old.y + beta.y * old.x + xi);
}

template <int KM>
__global__ void __launch_bounds__(SK_THREADS) skinny_kernel(const SkinnyDesc d, int chunk,
                                                            int beta_mode, float2 alpha_f) {
  extern __shared__ float4 s_sm[];  // [chunk][KM / 2]: two complex k per float4
  constexpr int KH = KM / 2;
  const long r = blockIdx.x * static_cast<long>(SK_THREADS) + threadIdx.x;
  const bool live = r < d.Mb;
  float2 g[KM];
  {
    const long go = live ? (d.gr ? d.gr[r] : r * d.ldg) : 0;
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      double2 x = make_double2(0.0, 0.0);
      if (live && k < d.K) x = d.G[go + (d.gk ? d.gk[k] : k * d.gks)];
      const float im = f64_to_f32(x.y);
      g[k] = make_float2(f64_to_f32(x.x), d.conjG ? -im : im);
    }
  }
  const long cb = live ? (d.cb ? d.cb[r] : r * d.ldcb) : 0;
  for (int s0 = 0; s0 < d.Ns; s0 += chunk) {
    const int ns = min(chunk, d.Ns - s0);
    __syncthreads();
    for (int i = threadIdx.x; i < ns * KH; i += SK_THREADS) {
      const int s = i / KH, kp = i - s * KH;
      const long so = d.sr ? d.sr[s0 + s] : static_cast<long>(s0 + s) * d.lds;
      const int k0 = 2 * kp, k1 = 2 * kp + 1;
      double2 x0 = make_double2(0.0, 0.0), x1 = make_double2(0.0, 0.0);
      if (k0 < d.K) x0 = d.S[so + (d.sk ? d.sk[k0] : k0 * d.sks)];
      if (k1 < d.K) x1 = d.S[so + (d.sk ? d.sk[k1] : k1 * d.sks)];
      const float sg = d.conjS ? -1.0f : 1.0f;
      s_sm[i] = make_float4(f64_to_f32(x0.x), sg * f64_to_f32(x0.y), f64_to_f32(x1.x),
                            sg * f64_to_f32(x1.y));
    }
    __syncthreads();
    if (!live) continue;
    // two outputs per pass; the old values of both are requested before the
    // products so their latency overlaps the arithmetic
    for (int s = 0; s < ns; s += 2) {
      const bool two = s + 1 < ns;
      const long co0 = cb + (d.cs ? d.cs[s0 + s] : static_cast<long>(s0 + s) * d.ldcs);
      const long co1 = two ? cb + (d.cs ? d.cs[s0 + s + 1] : static_cast<long>(s0 + s + 1) * d.ldcs)
                           : co0;
      // beta = 1 (one writer per element): the additions run in L2 as
      // atomics, with no read round trip; general beta reads the old values
      double2 old0 = make_double2(0.0, 0.0), old1 = make_double2(0.0, 0.0);
      if (beta_mode == 2) {
        old0 = d.C[co0];
        if (two) old1 = d.C[co1];
      }
      const float4 *q0 = s_sm + s * KH;
      const float4 *q1 = two ? q0 + KH : q0;
      float ar0 = 0.f, ai0 = 0.f, ar1 = 0.f, ai1 = 0.f;  // output s
      float br0 = 0.f, bi0 = 0.f, br1 = 0.f, bi1 = 0.f;  // output s + 1
#pragma unroll
      for (int kp = 0; kp < KH; ++kp) {
        const float4 w = q0[kp], u = q1[kp];
        const float2 a = g[2 * kp], b = g[2 * kp + 1];
        ar0 = fmaf(a.x, w.x, ar0);
        ar0 = fmaf(-a.y, w.y, ar0);
        ai0 = fmaf(a.x, w.y, ai0);
        ai0 = fmaf(a.y, w.x, ai0);
        ar1 = fmaf(b.x, w.z, ar1);
        ar1 = fmaf(-b.y, w.w, ar1);
        ai1 = fmaf(b.x, w.w, ai1);
        ai1 = fmaf(b.y, w.z, ai1);
        br0 = fmaf(a.x, u.x, br0);
        br0 = fmaf(-a.y, u.y, br0);
        bi0 = fmaf(a.x, u.y, bi0);
        bi0 = fmaf(a.y, u.x, bi0);
        br1 = fmaf(b.x, u.z, br1);
        br1 = fmaf(-b.y, u.w, br1);
        bi1 = fmaf(b.x, u.w, bi1);
        bi1 = fmaf(b.y, u.z, bi1);
      }
      if (beta_mode == 1) {
        const double2 x0 = epilogue(ar0 + ar1, ai0 + ai1, old0, alpha_f, 0, d.beta);
        atomicAdd(&d.C[co0].x, x0.x);
        atomicAdd(&d.C[co0].y, x0.y);
        if (two) {
          const double2 x1 = epilogue(br0 + br1, bi0 + bi1, old1, alpha_f, 0, d.beta);
          atomicAdd(&d.C[co1].x, x1.x);
          atomicAdd(&d.C[co1].y, x1.y);
        }
      } else {
        d.C[co0] = epilogue(ar0 + ar1, ai0 + ai1, old0, alpha_f, beta_mode, d.beta);
        if (two) d.C[co1] = epilogue(br0 + br1, bi0 + bi1, old1, alpha_f, beta_mode, d.beta);
      }
    }
  }
}

// FP64 variant (the FP64 tier and the Davidson subspace products): the
// same layout with FP64 operands and sums.
template <int KM>
__global__ void __launch_bounds__(SK_THREADS) skinny64_kernel(const SkinnyDesc d, int chunk) {
  extern __shared__ double2 s_sm64[];  // [chunk][KM]
  const long r = blockIdx.x * static_cast<long>(SK_THREADS) + threadIdx.x;
  const bool live = r < d.Mb;
  double2 g[KM];
  {
    const long go = live ? (d.gr ? d.gr[r] : r * d.ldg) : 0;
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      double2 x = make_double2(0.0, 0.0);
      if (live && k < d.K) x = d.G[go + (d.gk ? d.gk[k] : k * d.gks)];
      if (d.conjG) x.y = -x.y;
      g[k] = x;
    }
  }
  const long cb = live ? (d.cb ? d.cb[r] : r * d.ldcb) : 0;
  const bool b0 = d.beta.x == 0.0 && d.beta.y == 0.0;
  for (int s0 = 0; s0 < d.Ns; s0 += chunk) {
    const int ns = min(chunk, d.Ns - s0);
    __syncthreads();
    for (int i = threadIdx.x; i < ns * KM; i += SK_THREADS) {
      const int s = i / KM, k = i - s * KM;
      const long so = d.sr ? d.sr[s0 + s] : static_cast<long>(s0 + s) * d.lds;
      double2 x = make_double2(0.0, 0.0);
      if (k < d.K) x = d.S[so + (d.sk ? d.sk[k] : k * d.sks)];
      if (d.conjS) x.y = -x.y;
      s_sm64[i] = x;
    }
    __syncthreads();
    if (!live) continue;
    for (int s = 0; s < ns; ++s) {
      const long co = cb + (d.cs ? d.cs[s0 + s] : static_cast<long>(s0 + s) * d.ldcs);
      const double2 old = b0 ? make_double2(0.0, 0.0) : d.C[co];
      const double2 *q = s_sm64 + s * KM;
      double2 acc = make_double2(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < KM; ++k) acc = cfma(g[k], q[k], acc);
      const double2 x = cmul(d.alpha, acc);
      d.C[co] = b0 ? x : cadd(x, cmul(d.beta, old));
    }
  }
}

template <int KM>
void skinny_launch(const SkinnyDesc &d, cudaStream_t st) {
  // set once per process (thread-safe static initialisation)
  static const bool attr = [&] {
    CUDA_CHECK(cudaFuncSetAttribute(skinny_kernel<KM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    SK_SMEM));
    return true;
  }();
  (void)attr;
  const int per_s = (KM / 2) * static_cast<int>(sizeof(float4));
  const int chunk = std::max(1, std::min(d.Ns, SK_SMEM / per_s));
  const int beta_mode = (d.beta.x == 0.0 && d.beta.y == 0.0) ? 0
                        : (d.beta.x == 1.0 && d.beta.y == 0.0) ? 1
                                                               : 2;
  const float2 af = make_float2(static_cast<float>(d.alpha.x), static_cast<float>(d.alpha.y));
  const long blocks = (d.Mb + SK_THREADS - 1) / SK_THREADS;
  skinny_kernel<KM><<<static_cast<unsigned>(blocks), SK_THREADS, chunk * per_s, st>>>(d, chunk,
                                                                                     beta_mode, af);
  LAUNCH_CHECK();
  count_launch();
}

template <int KM>
void skinny64_launch(const SkinnyDesc &d, cudaStream_t st) {
  // set once per process (thread-safe static initialisation)
  static const bool attr = [&] {
    CUDA_CHECK(cudaFuncSetAttribute(skinny64_kernel<KM>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, SK_SMEM));
    return true;
  }();
  (void)attr;
  const int per_s = KM * static_cast<int>(sizeof(double2));
  const int chunk = std::max(1, std::min(d.Ns, SK_SMEM / per_s));
  const long blocks = (d.Mb + SK_THREADS - 1) / SK_THREADS;
  skinny64_kernel<KM><<<static_cast<unsigned>(blocks), SK_THREADS, chunk * per_s, st>>>(d, chunk);
  LAUNCH_CHECK();
  count_launch();
}

}  // namespace

void gemm_skinny(const SkinnyDesc &d, cudaStream_t st) {
  if (d.Mb <= 0 || d.Ns <= 0) return;
  if (d.K < 0 || d.K > SKINNY_MAX_K) fail(CC_ERR_ARG, "gemm_skinny: K out of range");
  if (d.Mb > 0x7fffffffL * SK_THREADS) fail(CC_ERR_ARG, "gemm_skinny: too many rows");
  if (d.f64) {
    if (d.K > SKINNY64_MAX_K) fail(CC_ERR_ARG, "gemm_skinny: K out of range (FP64)");
    if (d.K <= 8) skinny64_launch<8>(d, st);
    else if (d.K <= 16) skinny64_launch<16>(d, st);
    else if (d.K <= 24) skinny64_launch<24>(d, st);
    else skinny64_launch<32>(d, st);
    return;
  }
  if (d.K <= 16) skinny_launch<16>(d, st);
  else if (d.K <= 24) skinny_launch<24>(d, st);
  else if (d.K <= 32) skinny_launch<32>(d, st);
  else if (d.K <= 40) skinny_launch<40>(d, st);
  else skinny_launch<48>(d, st);
}

}  // namespace cdfns
