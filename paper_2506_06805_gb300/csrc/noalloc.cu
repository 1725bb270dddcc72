// cc_zgemm_noalloc: the complex GEMM of cc_zgemm_dev for callers that must
// not allocate device memory.
//
// Some callers cannot let a library call cudaMalloc: code running while a
// CUDA stream is being captured into a graph (allocation is not a capturable
// operation), host frameworks that hand out all device memory from their own
// pre-sized pool and treat any outside allocation as a leak or an
// out-of-memory risk, and latency-critical loops where a cudaMalloc would
// synchronise the device. For them this entry point keeps every temporary
// (the tensor-core operand planes and the error flag) in one fixed array in
// device global memory, declared below, so a call allocates nothing.
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
  if (tier < CC_TIER_FP64 || tier > CC_TIER_BF16X3 || M < 1 || N < 1 || K < 1 || !A || !B || !C)
    return CC_ERR_ARG;
  try {
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
