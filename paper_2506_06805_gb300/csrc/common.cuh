// Shared definitions for the CD/FNS IP-EOM-CCSD CUDA library.
//
// Complex numbers are stored interleaved (re, im): double2 for FP64 tensors,
// float2 for the FP32 staging planes of the tensor-core path.
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/cdfns.h"

namespace cdfns {

typedef double2 cplx;

__host__ __device__ inline cplx mk(double r, double i) { return make_double2(r, i); }
__host__ __device__ inline cplx cadd(cplx a, cplx b) { return mk(a.x + b.x, a.y + b.y); }
__host__ __device__ inline cplx csub(cplx a, cplx b) { return mk(a.x - b.x, a.y - b.y); }
__host__ __device__ inline cplx cmul(cplx a, cplx b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline cplx cconj(cplx a) { return mk(a.x, -a.y); }
__host__ __device__ inline cplx cscale(double s, cplx a) { return mk(s * a.x, s * a.y); }
__host__ __device__ inline cplx cfma(cplx a, cplx b, cplx c) {  // a*b + c
  c.x = fma(a.x, b.x, c.x); c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y); c.y = fma(a.y, b.x, c.y);
  return c;
}

// FP64 <-> FP32 conversions on the integer pipes. On GB300 the hardware
// conversion instructions run at the FP64 rate (about 2 per SM clock,
// measured), some 60x slower than FP32 or INT32 arithmetic, so every kernel
// that narrows FP64 operands or widens FP32 results uses these instead.
//
// Narrowing with round-to-nearest-even, bit-identical to __double2float_rn:
// the 52-bit mantissa keeps its top 23 bits and the 29 dropped bits decide
// the rounding (a carry out of the mantissa increments the exponent, and
// out of the largest exponent gives infinity, as IEEE 754 rounding does).
// Zeros are handled in place; results outside the FP32 normal range
// (denormals, infinities, NaN) take the hardware instruction.
__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const unsigned hi = static_cast<unsigned>(b >> 32), lo = static_cast<unsigned>(b);
  const unsigned e = (hi >> 20) & 0x7ffu;
  if (e - 897u <= 1150u - 897u) {
    unsigned f = (hi & 0x80000000u) | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rest = lo & 0x1fffffffu;
    f += (rest > 0x10000000u || (rest == 0x10000000u && (f & 1u))) ? 1u : 0u;
    return __uint_as_float(f);
  }
  if (((hi & 0x7fffffffu) | lo) == 0u) return __uint_as_float(hi & 0x80000000u);
  return __double2float_rn(x);
}

// Widening (exact): exponent rebiased by 1023 - 127, mantissa shifted into
// place. Zeros in place; FP32 denormals, infinities and NaN in hardware.
__device__ __forceinline__ double f32_to_f64(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned e = (u >> 23) & 0xffu;
  if (e - 1u <= 253u) {
    const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
    return __hiloint2double(static_cast<int>(hi), static_cast<int>(u << 29));
  }
  if ((u & 0x7fffffffu) == 0u) return __hiloint2double(static_cast<int>(u & 0x80000000u), 0);
  return static_cast<double>(x);
}

// Error raised inside the library; carries a CC_ERR_* code.
struct Error {
  int code;
  std::string msg;
};

[[noreturn]] void fail(int code, const std::string &msg);
void check_cuda(cudaError_t e, const char *what, const char *file, int line);
#define CUDA_CHECK(x) ::cdfns::check_cuda((x), #x, __FILE__, __LINE__)
#define LAUNCH_CHECK() ::cdfns::check_cuda(cudaGetLastError(), "kernel launch", __FILE__, __LINE__)

// Device workspace: every buffer the library owns goes through here so that
// the caller's allocator (for example PyTorch's caching allocator) can serve
// it. Buffers are freed when the Buf goes out of scope.
struct Allocator {
  void *(*alloc)(size_t, void *) = nullptr;
  void (*free)(void *, void *) = nullptr;
  void *user = nullptr;
  size_t in_use = 0;  // bytes currently held through this allocator
  size_t peak = 0;    // high-water mark of in_use
  size_t window = 0;  // high-water mark of in_use since the caller last set it
  size_t limit = 0;   // cap on in_use (0: none); a get() beyond it fails
  // While `recycle` is set (for the length of one library call, and only
  // without a limit), released blocks are kept here and handed to the next
  // request of the same size: the solvers allocate the same buffers in
  // every iteration, and each round trip through a caller's allocator
  // callback or cudaMalloc/cudaFree costs host time, cudaFree a device
  // synchronisation. Kept blocks do not count in in_use; a failed
  // allocation returns them all and tries once more.
  struct Held {
    void *p;
    size_t bytes;
    void (*fr)(void *, void *);
    void *fr_user;
  };
  std::vector<Held> held;
  size_t held_bytes = 0;
  bool recycle = false;
  void *get(size_t bytes);
  // release p (bytes long) through the functions that allocated it (the
  // allocator may have been replaced since)
  void put(void *p, size_t bytes, void (*fr)(void *, void *), void *fr_user);
  void flush_held();  // return every kept block
};
// Device bytes an allocation through `al` can still obtain: the driver's free
// memory less 2 GiB for work outside the allocator (library workspaces,
// fragmentation), plus, for a caller's caching allocator, the bytes this
// allocator has returned since its high-water mark (held in that cache);
// never more than the room left under al->limit.
size_t device_avail(const Allocator *al);

struct Buf {
  Allocator *al = nullptr;
  void *p = nullptr;
  size_t bytes = 0;
  void (*fr)(void *, void *) = nullptr;  // free function in force at allocation
  void *fr_user = nullptr;
  Buf() = default;
  Buf(Allocator *a, size_t n) { reset(a, n); }
  Buf(const Buf &) = delete;
  Buf &operator=(const Buf &) = delete;
  Buf(Buf &&o) noexcept { *this = std::move(o); }
  Buf &operator=(Buf &&o) noexcept {
    release();
    al = o.al; p = o.p; bytes = o.bytes; fr = o.fr; fr_user = o.fr_user;
    o.p = nullptr; o.bytes = 0;
    return *this;
  }
  ~Buf() { release(); }
  void reset(Allocator *a, size_t n);
  void release();
  template <class T> T *as() const { return reinterpret_cast<T *>(p); }
  cplx *c() const { return as<cplx>(); }
};

// Precision tiers of the contraction engine (CC_TIER_* in cdfns.h).
enum Tier {
  TIER_FP64 = 0,
  TIER_TF32 = 1,
  TIER_TF32X3 = 2,
  TIER_BF16X3 = 3,
  TIER_FP16 = 4,
  TIER_FP16X3 = 5
};
constexpr int TIER_LAST = TIER_FP16X3;
// Engine-internal, not a CC_TIER_*: the CUDA-core path with FP32 products
// (runs summed in FP64) in the kernels that have that form, FP64 elsewhere.
// Memory-bound matrix-vector shapes of the tensor-core tiers take it: the
// FP64 pipe of GB300 is far narrower than its memory.
constexpr int TIER_SIMT32 = 16;
// hi/lo operand planes, three products
__host__ __device__ inline bool tier_split(int t) {
  return t == TIER_TF32X3 || t == TIER_BF16X3 || t == TIER_FP16X3;
}
// FP16 planes scaled by fp16_scale() of the operand maximum
__host__ __device__ inline bool tier_scaled(int t) { return t == TIER_FP16 || t == TIER_FP16X3; }
// 2-byte plane elements (kind::f16), else 4-byte (kind::tf32)
__host__ __device__ inline bool tier_half(int t) { return t == TIER_BF16X3 || tier_scaled(t); }
// the accurate split tier of the same operand family
__host__ __device__ inline int tier_accurate(int t) {
  return t == TIER_FP64 ? TIER_FP64
         : tier_scaled(t) ? TIER_FP16X3
         : t == TIER_BF16X3 ? TIER_BF16X3
                            : TIER_TF32X3;
}

// Scale for the FP16 tier: the power of two 2^k with amax 2^k < 2^15, so
// every scaled magnitude stays below 2^15 (FP16 max 65504) and values down
// to amax 2^-29 remain normal numbers; 1 for amax = 0 or non-finite.
__host__ __device__ inline float fp16_scale(float amax) {
  if (!(amax > 0.0f) || !(amax < 3.0e38f)) return 1.0f;
  unsigned u;
#ifdef __CUDA_ARCH__
  u = __float_as_uint(amax);
#else
  std::memcpy(&u, &amax, sizeof(u));
#endif
  int k = 141 - static_cast<int>((u >> 23) & 0xffu);  // amax < 2^(eb - 126)
  k = k > 127 ? 127 : (k < -126 ? -126 : k);
  const unsigned r = static_cast<unsigned>(k + 127) << 23;
#ifdef __CUDA_ARCH__
  return __uint_as_float(r);
#else
  float f;
  std::memcpy(&f, &r, sizeof(f));
  return f;
#endif
}

// Kernel launch counters (for reporting how many kernels ran): the process
// total and the calling thread's own count.
extern std::atomic<unsigned long long> g_launches;
extern thread_local unsigned long long t_launches;
inline void count_launch(unsigned long long n = 1) {
  g_launches += n;
  t_launches += n;
}

}  // namespace cdfns
