// Host-side tensor contraction engine.
//
// contract(alpha, A, B, beta, C) computes
//   C[c-indices] = alpha * sum_{k} opA(A)[a-indices] opB(B)[b-indices] + beta * C
// for index strings such as "imae", "mbej" -> "ijab". Indices of C split
// into M (found in A) and N (found in B); indices in both A and B but not in C
// are contracted (K). The operands are addressed in place through offset
// tables (no permutation copies) for the FP64 GEMM, or packed once into the
// expanded real planes of the tensor-core GEMM for the fast tiers.
#pragma once

#include <map>
#include <set>
#include <string>
#include <vector>

#include "kernels.h"

namespace cdfns {

struct TRef {
  cplx *p = nullptr;
  std::string idx;
  std::vector<long> dims;
  std::vector<long> str;  // element strides
  bool conj = false;
  bool stable = false;  // contents fixed until Engine::clear_pack_cache()
  // FP16 tiers: device float >= max(|Re|, |Im|) over the whole tensor, when
  // the caller already has it (saves the operand's own maximum pass)
  const float *amax = nullptr;
  // output only: a device float that receives max(|Re|, |Im|) in FP32 over
  // the whole tensor once the contraction has written it (the view must be
  // the whole tensor); read by the next contraction's FP16 scale
  float *amax_out = nullptr;
  long size() const {
    long s = 1;
    for (long d : dims) s *= d;
    return s;
  }
};

// Contiguous row-major view.
TRef T(const cplx *p, const char *idx, std::initializer_list<long> dims, bool conj = false);
TRef T(const cplx *p, const std::string &idx, const std::vector<long> &dims, bool conj = false);
// Strided view.
TRef Tv(const cplx *p, const char *idx, std::initializer_list<long> dims,
        std::initializer_list<long> strides, bool conj = false);
inline TRef conj(TRef t) {
  t.conj = !t.conj;
  return t;
}
inline TRef with_amax(TRef t, const float *m) {
  t.amax = m;
  return t;
}
inline TRef with_amax_out(TRef t, float *m) {
  t.amax_out = m;
  return t;
}
// Whether a view addresses every element of its tensor exactly once
// (row-major strides of its dims and no repeated index letter): its
// maximum is then the maximum of the contiguous block.
bool whole_view(const TRef &t);
// Mark an operand whose contents stay fixed across calls (integrals, H-bar):
// its packed tensor-core planes are then built once and reused.
inline TRef stable(TRef t) {
  t.stable = true;
  return t;
}

class Engine {
 public:
  Allocator *al = nullptr;
  cudaStream_t st = nullptr;
  int num_sms = 148;
  int *err_flag = nullptr;  // device int, set by bounded waits
  // Device bytes to keep free when caching a stable operand's packed planes:
  // 0 caches every stable operand; otherwise an operand whose planes would
  // leave less free memory than this is packed into the scratch planes on
  // each use instead (the decision holds until the pack cache is cleared).
  size_t cache_reserve = 0;
  // statistics
  double flops = 0;
  long gen = 0;  // bumped whenever a plane or packed buffer is (re)allocated or freed

  void contract(cplx alpha, const TRef &A, const TRef &B, cplx beta, const TRef &C, int tier);
  // Same contraction prepared for a grouped launch (gemm_tc_grouped): packs
  // the operands into the planes of `slot` (distinct slots for contractions
  // launched together) and fills *out. Returns false when the contraction
  // was small or FP64 and has already run on the FP64 path.
  bool prepare(cplx alpha, const TRef &A, const TRef &B, cplx beta, const TRef &C, int tier,
               int slot, TcDesc *out);
  // out = alpha * permuted(in) + beta * out, where out's index string names
  // the order: e.g. permute_into(T(x,"ijab"), T(y,"jiab")) copies y with i,j
  // exchanged.
  void permute_into(cplx alpha, const TRef &in, cplx beta, const TRef &out);
  const long *table(const std::vector<long> &dims, const std::vector<long> &strides);
  // growable scratch planes for the tensor-core operands
  void *plane(int which, size_t bytes);
  void clear_cache() {
    cache_.clear();
    packs_.clear();
    uncached_.clear();
    ++gen;
  }
  void clear_pack_cache() {
    packs_.clear();
    uncached_.clear();
    ++gen;
  }
  // Drop the cached packed planes of the tensor at p: a tensor marked stable
  // for a stretch of work (the amplitudes within one residual) whose contents
  // change or whose memory is freed afterwards.
  void forget_packs(const void *p);

  // Optional device-time trace, on when the environment variable
  // CDFNS_TRACE names a file: every contraction (operand packing and GEMM)
  // and every region() scope is bracketed by CUDA events on the engine's
  // stream; trace_flush() waits for them and appends one CSV line per record
  // (label,M,N,K,tier,ms) to that file. Recording adds two event records per
  // contraction and nothing else.
  bool tracing() const { return trace_on_; }
  void trace_init();
  void trace_flush();
  struct Region {
    Engine *e;
    int rec;
    long epoch;  // records opened before a flush are not closed after it
    ~Region();
  };
  Region region(const std::string &label);

 private:
  struct Packed {
    Buf hi, lo, amax;
    const void *src = nullptr;
  };
  static std::string pack_key(bool a_side, const TRef &t, const long *rt, const long *kt, long ld,
                              long rows, long K, long Kp, int tier);
  // whether the packed planes of `key` (n bytes) are, or may be, cached
  bool may_cache(const std::string &key, size_t n);
  // returns (hi, lo) planes of a stable operand, packing it on first use;
  // *amax receives its FP16 scale source (TIER_FP16) or nullptr
  std::pair<void *, void *> packed(const std::string &key, bool a_side, const TRef &t,
                                   const long *rt, const long *kt, long ld, long rows, long K,
                                   long Kp, int tier, const float **amax, bool rows_unit);
  // device float of plane slot `which` for the FP16 operand maximum
  float *plane_amax(int which);
  std::map<int, Buf> amax_planes_;
  bool amax_done_ = false;  // the last contract() recorded C.amax_out in the GEMM epilogue
  std::map<std::string, Buf> cache_;
  std::map<std::string, Packed> packs_;
  std::set<std::string> uncached_;
  std::map<int, Buf> planes_;
  struct TraceRec {
    std::string label;
    long M, N, K;
    int tier;
    cudaEvent_t e0, e1;
    bool closed;
  };
  bool trace_on_ = false;
  std::string trace_path_;
  std::vector<TraceRec> trace_;
  long trace_epoch_ = 0;
  int trace_open(const std::string &label, long M, long N, long K, int tier);
  void trace_close(int rec);
  struct Plan;
  bool run(cplx alpha, const TRef &A, const TRef &B, cplx beta, const TRef &C, int tier, int slot,
           TcDesc *out);
};

inline cplx C1() { return mk(1.0, 0.0); }
inline cplx C0() { return mk(0.0, 0.0); }
inline cplx Cr(double r) { return mk(r, 0.0); }

}  // namespace cdfns
