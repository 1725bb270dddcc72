#include "engine.h"

#include <cstdio>
#include <cstdlib>

#include <algorithm>
#include <sstream>
#include <tuple>

namespace cdfns {

TRef T(const cplx *p, const std::string &idx, const std::vector<long> &dims, bool cj) {
  TRef t;
  t.p = const_cast<cplx *>(p);
  t.idx = idx;
  t.dims = dims;
  t.str.resize(dims.size());
  long s = 1;
  for (int i = static_cast<int>(dims.size()) - 1; i >= 0; --i) {
    t.str[i] = s;
    s *= dims[i];
  }
  t.conj = cj;
  if (idx.size() != dims.size()) fail(CC_ERR_ARG, "tensor view: index/dims mismatch " + idx);
  return t;
}

TRef T(const cplx *p, const char *idx, std::initializer_list<long> dims, bool cj) {
  return T(p, std::string(idx), std::vector<long>(dims), cj);
}

TRef Tv(const cplx *p, const char *idx, std::initializer_list<long> dims,
        std::initializer_list<long> strides, bool cj) {
  TRef t = T(p, idx, dims, cj);
  t.str = strides;
  if (t.str.size() != t.dims.size()) fail(CC_ERR_ARG, "strided view: rank mismatch");
  return t;
}

bool whole_view(const TRef &t) {
  long s = 1;
  for (int i = static_cast<int>(t.dims.size()) - 1; i >= 0; --i) {
    if (t.dims[i] != 1 && t.str[i] != s) return false;
    s *= t.dims[i];
  }
  for (size_t i = 0; i < t.idx.size(); ++i)
    for (size_t j = i + 1; j < t.idx.size(); ++j)
      if (t.idx[i] == t.idx[j]) return false;
  return true;
}

const long *Engine::table(const std::vector<long> &dims, const std::vector<long> &strides) {
  std::ostringstream key;
  for (size_t i = 0; i < dims.size(); ++i) key << dims[i] << ':' << strides[i] << ',';
  auto it = cache_.find(key.str());
  if (it != cache_.end()) return it->second.as<long>();
  long total = 1;
  for (long d : dims) total *= d;
  Buf b(al, sizeof(long) * std::max<long>(total, 1));
  make_offsets(b.as<long>(), static_cast<int>(dims.size()), dims.data(), strides.data(), st);
  const long *p = b.as<long>();
  cache_[key.str()] = std::move(b);
  return p;
}

std::string Engine::pack_key(bool a_side, const TRef &t, const long *rt, const long *kt, long ld,
                             long rows, long K, long Kp, int tier) {
  std::ostringstream key;
  key << (a_side ? 'A' : 'B') << t.p << ':' << t.conj << ':' << rt << ':' << kt << ':' << ld << ':'
      << rows << ':' << K << ':' << Kp << ':' << tier;
  return key.str();
}

bool Engine::may_cache(const std::string &key, size_t n) {
  if (cache_reserve == 0 || packs_.count(key)) return true;
  if (uncached_.count(key)) return false;
  if (device_avail(al) >= n + cache_reserve) return true;
  uncached_.insert(key);
  return false;
}

std::pair<void *, void *> Engine::packed(const std::string &key, bool a_side, const TRef &t,
                                         const long *rt, const long *kt, long ld, long rows, long K,
                                         long Kp, int tier, const float **amax, bool rows_unit) {
  auto it = packs_.find(key);
  if (it != packs_.end()) {
    *amax = it->second.amax.as<float>();
    return {it->second.hi.p, it->second.lo.p};
  }
  const size_t eb = tc_elem_bytes(tier);
  const size_t n = eb * (a_side ? 2 : 1) * rows * Kp;
  Packed pk;
  ++gen;
  pk.src = t.p;
  pk.hi.reset(al, n);
  if (tier_split(tier)) pk.lo.reset(al, n);
  if (tier_scaled(tier)) {
    pk.amax.reset(al, sizeof(float));
    if (t.amax)
      CUDA_CHECK(cudaMemcpyAsync(pk.amax.p, t.amax, sizeof(float), cudaMemcpyDeviceToDevice, st));
    else if (whole_view(t))
      tc_absmax(t.p, nullptr, nullptr, 0, 1, t.size(), pk.amax.as<float>(), st);
    else
      tc_absmax(t.p, rt, kt, ld, rows, K, pk.amax.as<float>(), st);
  }
  if (a_side)
    tc_pack_A(t.p, rt, kt, ld, t.conj, rows, K, Kp, tier, pk.hi.p, pk.lo.p, st, pk.amax.as<float>(),
              rows_unit);
  else
    tc_pack_B(t.p, rt, kt, ld, t.conj, rows, K, Kp, tier, pk.hi.p, pk.lo.p, st, pk.amax.as<float>(),
              rows_unit);
  std::pair<void *, void *> r{pk.hi.p, pk.lo.p};
  *amax = pk.amax.as<float>();
  packs_[key] = std::move(pk);
  return r;
}

void Engine::forget_packs(const void *p) {
  bool any = false;
  for (auto it = packs_.begin(); it != packs_.end();) {
    if (it->second.src == p) {
      it = packs_.erase(it);
      any = true;
    } else {
      ++it;
    }
  }
  std::ostringstream a, b;
  a << 'A' << p << ':';
  b << 'B' << p << ':';
  for (auto it = uncached_.begin(); it != uncached_.end();) {
    if (it->compare(0, a.str().size(), a.str()) == 0 || it->compare(0, b.str().size(), b.str()) == 0)
      it = uncached_.erase(it);
    else
      ++it;
  }
  if (any) ++gen;
}

float *Engine::plane_amax(int which) {
  Buf &b = amax_planes_[which];
  if (!b.p) {
    b.reset(al, sizeof(float));
    ++gen;
  }
  return b.as<float>();
}

void *Engine::plane(int which, size_t bytes) {
  Buf &b = planes_[which];
  if (b.bytes < bytes) {
    b.release();
    b.reset(al, bytes + bytes / 8);
    ++gen;
  }
  return b.p;
}

namespace {

int find(const std::string &s, char c) {
  const size_t p = s.find(c);
  return p == std::string::npos ? -1 : static_cast<int>(p);
}

// A table that is a plain linear map (offset = i * step) is not needed.
bool linear(const std::vector<long> &dims, const std::vector<long> &str, long *step) {
  // row-major contiguous block with a uniform inner stride
  if (dims.empty()) {
    *step = 0;
    return true;
  }
  long expect = str.back();
  for (int i = static_cast<int>(dims.size()) - 1; i >= 0; --i) {
    if (dims[i] == 1) continue;
    if (str[i] != expect) return false;
    expect *= dims[i];
  }
  *step = str.back();
  // if every dim of size 1 the step is irrelevant
  return true;
}

}  // namespace

void Engine::contract(cplx alpha, const TRef &A, const TRef &B, cplx beta, const TRef &C,
                      int tier) {
  if (C.amax_out && !whole_view(C))
    fail(CC_ERR_ARG, "contract: an output maximum needs the whole output tensor as the view");
  amax_done_ = false;
  run(alpha, A, B, beta, C, tier, -1, nullptr);
  // the tensor-core epilogue records it for plain stores; otherwise one pass
  if (C.amax_out && !amax_done_) tc_absmax(C.p, nullptr, nullptr, 0, 1, C.size(), C.amax_out, st);
}

bool Engine::prepare(cplx alpha, const TRef &A, const TRef &B, cplx beta, const TRef &C, int tier,
                     int slot, TcDesc *out) {
  if (slot < 0 || !out) fail(CC_ERR_ARG, "prepare: slot and descriptor required");
  if (C.amax_out) fail(CC_ERR_ARG, "prepare: output maxima are not tracked in grouped launches");
  return run(alpha, A, B, beta, C, tier, slot, out);
}

void Engine::trace_init() {
  const char *p = std::getenv("CDFNS_TRACE");
  trace_on_ = p && p[0];
  if (trace_on_) trace_path_ = p;
}

int Engine::trace_open(const std::string &label, long M, long N, long K, int tier) {
  if (!trace_on_) return -1;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cap);
  if (cap != cudaStreamCaptureStatusNone) return -1;
  TraceRec r{label, M, N, K, tier, nullptr, nullptr, false};
  CUDA_CHECK(cudaEventCreate(&r.e0));
  CUDA_CHECK(cudaEventCreate(&r.e1));
  CUDA_CHECK(cudaEventRecord(r.e0, st));
  trace_.push_back(r);
  return static_cast<int>(trace_.size()) - 1;
}

void Engine::trace_close(int rec) {
  if (rec < 0 || rec >= static_cast<int>(trace_.size())) return;
  CUDA_CHECK(cudaEventRecord(trace_[rec].e1, st));
  trace_[rec].closed = true;
}

Engine::Region Engine::region(const std::string &label) {
  return Region{this, trace_open(label, 0, 0, 0, -1), trace_epoch_};
}

Engine::Region::~Region() {
  if (rec >= 0 && epoch == e->trace_epoch_) e->trace_close(rec);
}

void Engine::trace_flush() {
  if (!trace_on_ || trace_.empty()) return;
  FILE *f = std::fopen(trace_path_.c_str(), "a");
  for (TraceRec &r : trace_) {
    float ms = -1.0f;
    if (r.closed && cudaEventSynchronize(r.e1) == cudaSuccess &&
        cudaEventElapsedTime(&ms, r.e0, r.e1) != cudaSuccess)
      ms = -1.0f;
    if (f && r.closed)
      std::fprintf(f, "%s,%ld,%ld,%ld,%d,%.4f\n", r.label.c_str(), r.M, r.N, r.K, r.tier,
                   static_cast<double>(ms));
    cudaEventDestroy(r.e0);
    cudaEventDestroy(r.e1);
  }
  if (f) std::fclose(f);
  cudaGetLastError();
  trace_.clear();
  ++trace_epoch_;
}

bool Engine::run(cplx alpha, const TRef &A, const TRef &B, cplx beta, const TRef &C, int tier,
                 int slot, TcDesc *out) {
  std::vector<long> mdim, amstr, cmstr, ndim, bnstr, cnstr, kdim, akstr, bkstr;
  for (size_t i = 0; i < C.idx.size(); ++i) {
    const char c = C.idx[i];
    const int ia = find(A.idx, c), ib = find(B.idx, c);
    if (ia >= 0 && ib >= 0) fail(CC_ERR_ARG, std::string("contract: batch index ") + c);
    if (ia >= 0) {
      if (A.dims[ia] != C.dims[i]) fail(CC_ERR_ARG, std::string("contract: dim mismatch ") + c);
      mdim.push_back(C.dims[i]);
      amstr.push_back(A.str[ia]);
      cmstr.push_back(C.str[i]);
    } else if (ib >= 0) {
      if (B.dims[ib] != C.dims[i]) fail(CC_ERR_ARG, std::string("contract: dim mismatch ") + c);
      ndim.push_back(C.dims[i]);
      bnstr.push_back(B.str[ib]);
      cnstr.push_back(C.str[i]);
    } else {
      fail(CC_ERR_ARG, std::string("contract: output index not in inputs ") + c);
    }
  }
  for (size_t i = 0; i < A.idx.size(); ++i) {
    const char c = A.idx[i];
    if (find(C.idx, c) >= 0) continue;
    const int ib = find(B.idx, c);
    if (ib < 0) fail(CC_ERR_ARG, std::string("contract: dangling index ") + c);
    if (A.dims[i] != B.dims[ib]) fail(CC_ERR_ARG, std::string("contract: K dim mismatch ") + c);
    kdim.push_back(A.dims[i]);
    akstr.push_back(A.str[i]);
    bkstr.push_back(B.str[ib]);
  }
  for (size_t i = 0; i < B.idx.size(); ++i) {
    const char c = B.idx[i];
    if (find(C.idx, c) < 0 && find(A.idx, c) < 0)
      fail(CC_ERR_ARG, std::string("contract: dangling index ") + c);
  }
  long M = 1, N = 1, K = 1;
  for (long d : mdim) M *= d;
  for (long d : ndim) N *= d;
  for (long d : kdim) K *= d;
  if (M == 0 || N == 0) return false;
  flops += 8.0 * M * N * K;
  const bool tiny = static_cast<double>(M) * N * K < 2.0e6 || K < 16 || M < 8 || N < 8;
  const bool simt = tier == TIER_FP64 || tier == TIER_SIMT32 || tiny;
  if (simt && (M == 1 || N == 1)) {
    // matrix-vector shape: order the outputs by decreasing stride in the
    // matrix operand, so that neighbouring threads read neighbouring elements
    // (each output's own sum over k is unchanged)
    std::vector<long> &d = N == 1 ? mdim : ndim, &s = N == 1 ? amstr : bnstr,
                      &c = N == 1 ? cmstr : cnstr;
    std::vector<size_t> ord(d.size());
    for (size_t i = 0; i < ord.size(); ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](size_t x, size_t y) { return s[x] > s[y]; });
    std::vector<long> d2, s2, c2;
    for (size_t i : ord) {
      d2.push_back(d[i]);
      s2.push_back(s[i]);
      c2.push_back(c[i]);
    }
    d.swap(d2);
    s.swap(s2);
    c.swap(c2);
  }
  // Tensor-core products with a long K: when an operand's K is strided but
  // one of its free indices has unit stride, that index becomes the fastest
  // of the GEMM rows, so the operand is packed by the transposing kernel
  // (reads along its rows) instead of by strided gathers. The output is then
  // written in a less regular order, which costs little against the long
  // accumulation of each tile.
  const bool skinny_shape = K <= SKINNY_MAX_K && std::min(M, N) <= 1024 && std::max(M, N) >= 2048;
  static const long rows_min_k = [] {
    // smallest K for the reordering; CDFNS_ROWS_MIN_K (read once) replaces
    // it, for tuning and for checking this path at small sizes
    const char *e = std::getenv("CDFNS_ROWS_MIN_K");
    return e ? std::atol(e) : 4096L;
  }();
  if (!simt && !skinny_shape && K >= rows_min_k) {
    auto unit_last = [](std::vector<long> &d, std::vector<long> &s, std::vector<long> &c,
                        const std::vector<long> &ks) {
      if (d.size() < 2 || s.back() == 1 || ks.empty() || ks.back() == 1) return;
      for (size_t u = 0; u + 1 < d.size(); ++u) {
        if (s[u] != 1) continue;
        std::rotate(d.begin() + u, d.begin() + u + 1, d.end());
        std::rotate(s.begin() + u, s.begin() + u + 1, s.end());
        std::rotate(c.begin() + u, c.begin() + u + 1, c.end());
        return;
      }
    };
    unit_last(mdim, amstr, cmstr, akstr);
    unit_last(ndim, bnstr, cnstr, bkstr);
  }
  const int trec =
      trace_on_ ? trace_open((out ? "prep " : "") + A.idx + (A.conj ? "*" : "") + "," + B.idx +
                                 (B.conj ? "*" : "") + "->" + C.idx,
                             M, N, K, tiny ? 0 : tier)
                : -1;
  Region closer{this, trec, trace_epoch_};

  // tables (NULL when linear)
  long step;
  const long *am = nullptr, *ak = nullptr, *bn = nullptr, *bk = nullptr, *cm = nullptr, *cn = nullptr;
  long lda = 0, ldb = 0, ldc = 0;
  if (linear(mdim, amstr, &step)) lda = step; else am = table(mdim, amstr);
  if (linear(mdim, cmstr, &step)) ldc = step; else cm = table(mdim, cmstr);
  if (linear(ndim, bnstr, &step)) ldb = step; else bn = table(ndim, bnstr);
  {
    long s2;
    if (!(linear(ndim, cnstr, &s2) && s2 == 1 && !ndim.empty())) {
      if (ndim.empty()) {
        cn = nullptr;  // N = 1: offset 0
      } else {
        cn = table(ndim, cnstr);
      }
    }
  }
  if (!(linear(kdim, akstr, &step) && (kdim.empty() || step == 1))) ak = table(kdim, akstr);
  if (!(linear(kdim, bkstr, &step) && (kdim.empty() || step == 1))) bk = table(kdim, bkstr);
  if (mdim.empty()) { lda = 0; ldc = 0; }
  if (ndim.empty()) ldb = 0;

  // small or skinny products stay on the CUDA-core path (GEMV or a few tiles)
  if (simt) {
    GemmDesc g;
    g.M = M; g.N = N; g.K = K;
    g.A = A.p; g.am = am; g.ak = ak; g.lda = lda; g.conjA = A.conj;
    g.B = B.p; g.bn = bn; g.bk = bk; g.ldb = ldb; g.conjB = B.conj;
    g.C = C.p; g.cm = cm; g.cn = cn; g.ldc = ldc;
    g.alpha = alpha; g.beta = beta;
    g.k_contig = kdim.empty() || (M == 1 ? bkstr.back() == 1 : akstr.back() == 1);
    g.f32 = tier != TIER_FP64;
    gemm_f64(g, st, num_sms);
    return false;
  }
  // short contracted index with one short free side: FP32 on the CUDA cores
  if (K <= SKINNY_MAX_K && std::min(M, N) <= 1024 && std::max(M, N) >= 2048) {
    SkinnyDesc d;
    d.K = static_cast<int>(K);
    d.alpha = alpha;
    d.beta = beta;
    d.C = C.p;
    const long *ak_ = kdim.empty() ? nullptr : ak, *bk_ = kdim.empty() ? nullptr : bk;
    if (N <= M) {  // long side A (rows m), short side B (rows n)
      d.Mb = M; d.Ns = static_cast<int>(N);
      d.G = A.p; d.gr = am; d.ldg = lda; d.gk = ak_; d.conjG = A.conj;
      d.S = B.p; d.sr = bn; d.lds = ldb; d.sk = bk_; d.conjS = B.conj;
      d.cb = cm; d.ldcb = ldc; d.cs = cn; d.ldcs = 1;
    } else {       // long side B (rows n), short side A (rows m)
      d.Mb = N; d.Ns = static_cast<int>(M);
      d.G = B.p; d.gr = bn; d.ldg = ldb; d.gk = bk_; d.conjG = B.conj;
      d.S = A.p; d.sr = am; d.lds = lda; d.sk = ak_; d.conjS = A.conj;
      d.cb = cn; d.ldcb = 1; d.cs = cm; d.ldcs = ldc;
    }
    gemm_skinny(d, st);
    return false;
  }
  // fast tier: pack operands into expanded planes, tensor-core GEMM
  const int kal = tc_k_align(tier);
  const long Kp = ((2 * K + kal - 1) / kal) * kal;
  const size_t eb = tc_elem_bytes(tier);
  const bool split = tier_split(tier);
  void *Ah, *Al = nullptr, *Bh, *Bl = nullptr;
  const int pb = 4 * (slot < 0 ? 0 : slot + 1);  // plane set of this contraction
  const bool f16 = tier_scaled(tier);
  const float *xa = nullptr, *xb = nullptr;  // FP16 operand maxima
  const size_t nA_bytes = eb * 2 * M * Kp * (split ? 2 : 1), nB_bytes = eb * N * Kp * (split ? 2 : 1);
  // read along rows (transposing through shared memory) when k is strided
  // but neighbouring rows are neighbouring elements
  const bool a_rows = !mdim.empty() && amstr.back() == 1 && !kdim.empty() && akstr.back() != 1;
  const bool b_rows = !ndim.empty() && bnstr.back() == 1 && !kdim.empty() && bkstr.back() != 1;
  std::string keyA, keyB;
  if (A.stable) keyA = pack_key(true, A, am, ak, lda, M, K, Kp, tier);
  if (B.stable) keyB = pack_key(false, B, bn, bk, ldb, N, K, Kp, tier);
  if (A.stable && may_cache(keyA, nA_bytes)) {
    std::tie(Ah, Al) = packed(keyA, true, A, am, ak, lda, M, K, Kp, tier, &xa, a_rows);
  } else {
    Ah = plane(pb + 0, eb * 2 * M * Kp);
    Al = split ? plane(pb + 1, eb * 2 * M * Kp) : nullptr;
    Region r = region("pack A " + A.idx);
    if (f16 && A.amax) {
      xa = A.amax;
    } else if (f16) {
      float *x = plane_amax(pb + 0);
      if (whole_view(A))
        tc_absmax(A.p, nullptr, nullptr, 0, 1, A.size(), x, st);
      else
        tc_absmax(A.p, am, ak, lda, M, K, x, st);
      xa = x;
    }
    tc_pack_A(A.p, am, ak, lda, A.conj, M, K, Kp, tier, Ah, Al, st, xa, a_rows);
  }
  if (B.stable && may_cache(keyB, nB_bytes)) {
    std::tie(Bh, Bl) = packed(keyB, false, B, bn, bk, ldb, N, K, Kp, tier, &xb, b_rows);
  } else {
    Bh = plane(pb + 2, eb * N * Kp);
    Bl = split ? plane(pb + 3, eb * N * Kp) : nullptr;
    Region r = region("pack B " + B.idx);
    if (f16 && B.amax) {
      xb = B.amax;
    } else if (f16) {
      float *x = plane_amax(pb + 2);
      if (whole_view(B))
        tc_absmax(B.p, nullptr, nullptr, 0, 1, B.size(), x, st);
      else
        tc_absmax(B.p, bn, bk, ldb, N, K, x, st);
      xb = x;
    }
    tc_pack_B(B.p, bn, bk, ldb, B.conj, N, K, Kp, tier, Bh, Bl, st, xb, b_rows);
  }
  TcDesc t;
  t.M = M; t.N = N; t.Kp = Kp;
  t.A = Ah; t.Alo = Al; t.B = Bh; t.Blo = Bl;
  t.tier = tier;
  t.C = C.p; t.cm = cm; t.cn = cn; t.ldc = ldc;
  t.alpha = alpha; t.beta = beta;
  t.amax_a = xa; t.amax_b = xb;
  t.bn = tc_pick_bn(N);
  const long tiles = ((2 * M + 127) / 128) * ((N + t.bn - 1) / t.bn);
  const int sk = tc_pick_split(tiles, Kp / kal, num_sms);
  t.split_k = sk;
  if (sk > 1) {
    scale_2d(C.p, cm, cn, ldc, M, N, beta, st);
    t.out = TC_OUT_F64_ATOMIC;
  } else {
    t.out = TC_OUT_F64;
  }
  if (out) {
    *out = t;
    return true;
  }
  if (C.amax_out && t.out == TC_OUT_F64 && beta.x == 0.0 && beta.y == 0.0) {
    CUDA_CHECK(cudaMemsetAsync(C.amax_out, 0, sizeof(float), st));
    t.amax_out = C.amax_out;
    t.amax_mul = 1.0f;
    amax_done_ = true;
  }
  Region r = region("gemm " + A.idx + "," + B.idx + "->" + C.idx);
  gemm_tc(t, st, err_flag);
  return false;
}

void Engine::permute_into(cplx alpha, const TRef &in, cplx beta, const TRef &out) {
  Region r = region("permute " + in.idx + "->" + out.idx);
  // out must be contiguous; in strides reordered to out's index order
  std::vector<long> istr(out.idx.size());
  for (size_t i = 0; i < out.idx.size(); ++i) {
    const int p = find(in.idx, out.idx[i]);
    if (p < 0 || in.dims[p] != out.dims[i]) fail(CC_ERR_ARG, "permute_into: index mismatch");
    istr[i] = in.str[p];
  }
  long expect = 1;
  for (int i = static_cast<int>(out.dims.size()) - 1; i >= 0; --i) {
    if (out.str[i] != expect && out.dims[i] != 1) fail(CC_ERR_ARG, "permute_into: out not contiguous");
    expect *= out.dims[i];
  }
  permute(out.p, in.p, static_cast<int>(out.dims.size()), out.dims.data(), istr.data(), alpha, beta,
          in.conj != out.conj, st);
}

}  // namespace cdfns
