// cc_zgemm_noalloc: the complex GEMM of cc_zgemm_dev for callers that must
// not allocate device memory.
//
// Some callers cannot let a library call cudaMalloc: host frameworks that
// reserve nearly all device memory up front for their own pool, where an
// outside allocation either fails or eats into memory the framework has
// promised elsewhere; applications whose device-memory budget is fixed at
// start-up and audited; and latency-critical loops, where cudaMalloc and
// cudaFree can synchronise the device and stall the pipeline. For them this
// entry point keeps every temporary (the tensor-core operand planes and the
// error flag) in one fixed array in device global memory, declared below, so
// a call allocates nothing and calls no allocating library routine.
//
// The array has a fixed size (kScratchBytes); every GPU that loads this
// library holds it until the process exits. All calls share it: it keeps the
// last call's contents, and two calls whose work overlaps on the GPU (for
// example on two streams) race on it, so callers must order them.
#include <mutex>
#include <string>

#include "kernels.h"

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;  // 64 MiB
constexpr size_t kFlagBytes = 256;                  // error flag region

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch for each device, looked up once per device
// with that device current (the host-side name is only a stand-in).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {nullptr};

void *scratch_for_current_device() {
  int dev = 0;
  CUDA_CHECK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) cdfns::fail(CC_ERR_UNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      cdfns::fail(CC_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch) failed: ") +
                                   cudaGetErrorString(e));
    }
    g_addr[dev] = p;
  }
  return g_addr[dev];
}

size_t round256(size_t n) { return (n + 255) & ~size_t(255); }

}  // namespace

namespace cdfns {
cudaStream_t noalloc_stream();                    // the process-wide default stream
void noalloc_record_error(const std::string &m);  // message for cc_last_error(NULL)
}

extern "C" int cc_zgemm_noalloc(int tier, long M, long N, long K, const double *A, const double *B,
                                double *C) {
  using namespace cdfns;
  try {
    if (tier < CC_TIER_FP64 || tier > CC_TIER_FP16X3)
      fail(CC_ERR_ARG, "cc_zgemm_noalloc: unknown tier " + std::to_string(tier));
    if (tier == CC_TIER_FP16 || tier == CC_TIER_FP16X3)
      fail(CC_ERR_ARG,
           "cc_zgemm_noalloc: the FP16 tiers need device scratch for their operand scales; "
           "use CC_TIER_FP64, CC_TIER_TF32, CC_TIER_TF32X3 or CC_TIER_BF16X3");
    if (M < 1 || N < 1 || K < 1 || !A || !B || !C)
      fail(CC_ERR_ARG, "cc_zgemm_noalloc: sizes must be >= 1 and pointers non-NULL");
    // byte extents of A, B and C (16 bytes per complex element) must be
    // representable, so no size computed below can wrap around
    long bytes = 0;
    if (__builtin_mul_overflow(M, K, &bytes) || __builtin_mul_overflow(bytes, 16L, &bytes) ||
        __builtin_mul_overflow(N, K, &bytes) || __builtin_mul_overflow(bytes, 16L, &bytes) ||
        __builtin_mul_overflow(M, N, &bytes) || __builtin_mul_overflow(bytes, 16L, &bytes))
      fail(CC_ERR_ARG, "cc_zgemm_noalloc: M, N, K too large (byte sizes overflow)");
    cudaStream_t st = noalloc_stream();
    const cplx *a = reinterpret_cast<const cplx *>(A);
    const cplx *b = reinterpret_cast<const cplx *>(B);
    cplx *c = reinterpret_cast<cplx *>(C);
    if (tier == CC_TIER_FP64) {
      // the FP64 path needs no temporaries for contiguous operands
      GemmDesc g;
      g.M = M; g.N = N; g.K = K;
      g.A = a; g.lda = K;
      g.B = b; g.ldb = K;
      g.C = c; g.ldc = N;
      int dev = 0, sms = 148;
      CUDA_CHECK(cudaGetDevice(&dev));
      CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      gemm_f64(g, st, sms);
      CUDA_CHECK(cudaStreamSynchronize(st));
      return CC_OK;
    }
    // every operand plane needs at least one byte per row and K element:
    // anything larger than the array is refused before sizing the planes
    if (M > static_cast<long>(kScratchBytes) || N > static_cast<long>(kScratchBytes) ||
        K > static_cast<long>(kScratchBytes))
      fail(CC_ERR_ARG, "cc_zgemm_noalloc: operands exceed the fixed " +
                           std::to_string(kScratchBytes) + "-byte scratch array");
    const int kal = tc_k_align(tier);
    const long Kp = ((2 * K + kal - 1) / kal) * kal;
    const size_t eb = tc_elem_bytes(tier);
    const bool split = tier != CC_TIER_TF32;
    const size_t a_bytes = round256(eb * 2 * static_cast<size_t>(M) * Kp);
    const size_t b_bytes = round256(eb * static_cast<size_t>(N) * Kp);
    const size_t need = kFlagBytes + (split ? 2 : 1) * (a_bytes + b_bytes);
    if (need > kScratchBytes) {
      fail(CC_ERR_ARG, "cc_zgemm_noalloc: operands need " + std::to_string(need) +
                           " bytes of scratch, more than the fixed " +
                           std::to_string(kScratchBytes) + " bytes");
    }
    unsigned char *base = static_cast<unsigned char *>(scratch_for_current_device());
    int *err = reinterpret_cast<int *>(base);
    unsigned char *p = base + kFlagBytes;
    void *Ah = p;
    p += a_bytes;
    void *Bh = p;
    p += b_bytes;
    void *Al = split ? static_cast<void *>(p) : nullptr;
    if (split) p += a_bytes;
    void *Bl = split ? static_cast<void *>(p) : nullptr;
    CUDA_CHECK(cudaMemsetAsync(err, 0, sizeof(int), st));  // the flag must start at zero
    tc_pack_A(a, nullptr, nullptr, K, false, M, K, Kp, tier, Ah, Al, st);
    tc_pack_B(b, nullptr, nullptr, K, false, N, K, Kp, tier, Bh, Bl, st);
    TcDesc t;
    t.M = M; t.N = N; t.Kp = Kp;
    t.A = Ah; t.Alo = Al; t.B = Bh; t.Blo = Bl;
    t.tier = tier;
    t.out = TC_OUT_F64;
    t.C = c; t.ldc = N;
    t.split_k = 1;
    t.no_tune = true;  // the tile autotuner would allocate; cached choices only
    gemm_tc(t, st, err);
    int h = 0;
    CUDA_CHECK(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaStreamSynchronize(st));
    if (h) fail(CC_ERR_TIMEOUT, "cc_zgemm_noalloc: a bounded device wait expired");
    return CC_OK;
  } catch (const Error &e) {
    noalloc_record_error(e.msg);
    return e.code;
  }
}
