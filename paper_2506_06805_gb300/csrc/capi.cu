// extern "C" boundary of libcdfns.so (declared in include/cdfns.h).
#include <algorithm>
#include <cstring>
#include <mutex>

#include "solver.h"

namespace cdfns {

namespace {
std::mutex g_mu;
std::string g_last_error;
Allocator g_default_alloc;
cudaStream_t g_default_stream = nullptr;
}  // namespace

void fail(int code, const std::string &msg) { throw Error{code, msg}; }

cudaStream_t noalloc_stream() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_default_stream;
}

void noalloc_record_error(const std::string &m) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_last_error = m;
}

void check_cuda(cudaError_t e, const char *what, const char *file, int line) {
  if (e == cudaSuccess) return;
  const int code = (e == cudaErrorMemoryAllocation) ? CC_ERR_OOM : CC_ERR_CUDA;
  fail(code, std::string(what) + ": " + cudaGetErrorString(e) + " (" + file + ":" +
                 std::to_string(line) + ")");
}

void *Allocator::get(size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (limit && in_use + bytes > limit)
    fail(CC_ERR_OOM, "device allocation of " + std::to_string(bytes) +
                         " bytes exceeds the context's memory limit");
  void *p = nullptr;
  for (size_t i = held.size(); i-- > 0;) {
    const Held &h = held[i];
    if (h.bytes == bytes && h.fr == free && h.fr_user == user) {
      p = h.p;
      held_bytes -= bytes;
      held.erase(held.begin() + static_cast<long>(i));
      break;
    }
  }
  for (int attempt = 0; !p; ++attempt) {
    if (alloc) {
      p = alloc(bytes, user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    if (p) break;
    if (attempt == 0 && !held.empty()) {
      flush_held();  // the kept blocks back to their allocator, then once more
      continue;
    }
    fail(CC_ERR_OOM, (alloc ? "device allocation of " : "cudaMalloc of ") +
                         std::to_string(bytes) + " bytes failed");
  }
  in_use += bytes;
  peak = std::max(peak, in_use);
  window = std::max(window, in_use);
  return p;
}

void Allocator::put(void *p, size_t bytes, void (*fr)(void *, void *), void *fr_user) {
  if (!p) return;
  const size_t n = bytes ? bytes : size_t(16);
  in_use -= std::min(in_use, n);
  if (recycle && limit == 0) {
    held.push_back(Held{p, n, fr, fr_user});
    held_bytes += n;
    return;
  }
  if (fr) fr(p, fr_user);
  else cudaFree(p);
}

void Allocator::flush_held() {
  for (const Held &h : held) {
    if (h.fr) h.fr(h.p, h.fr_user);
    else cudaFree(h.p);
  }
  held.clear();
  held_bytes = 0;
}

size_t device_avail(const Allocator *al) {
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    fr = 0;
  }
  const size_t reserve = size_t(2) << 30;
  fr = fr > reserve ? fr - reserve : 0;
  // (blocks kept for reuse are part of that difference; with cudaMalloc
  // they are added here, as a failed allocation returns them first)
  if (al && al->alloc) fr += al->peak - std::min(al->peak, al->in_use);
  else if (al) fr += al->held_bytes;
  if (al && al->limit) fr = std::min(fr, al->limit - std::min(al->limit, al->in_use));
  return fr;
}

void Buf::reset(Allocator *a, size_t n) {
  release();
  al = a;
  p = a->get(n);
  bytes = n;
  fr = a->free;
  fr_user = a->user;
}

void Buf::release() {
  if (p && al) al->put(p, bytes, fr, fr_user);
  p = nullptr;
  bytes = 0;
}

}  // namespace cdfns

using cdfns::Ctx;
using cdfns::Error;

namespace {

// For the length of one call, blocks the context releases are kept for
// reuse by its next requests of the same size; all are returned at the end.
struct RecycleScope {
  cdfns::Allocator *al;
  bool was;
  explicit RecycleScope(cc_ctx *ctx) : al(ctx ? &ctx->c.al : nullptr), was(al && al->recycle) {
    if (al) al->recycle = true;
  }
  ~RecycleScope() {
    if (!al || was) return;
    al->recycle = false;
    try {
      al->flush_held();
    } catch (...) {
    }
  }
};

template <class F>
int guarded(cc_ctx *ctx, F &&f) {
  RecycleScope recycle(ctx);
  try {
    return f();
  } catch (const Error &e) {
    if (ctx) ctx->c.last_error = e.msg;
    std::lock_guard<std::mutex> lk(cdfns::g_mu);
    cdfns::g_last_error = e.msg;
    return e.code;
  } catch (const std::bad_alloc &) {
    if (ctx) ctx->c.last_error = "host allocation failed";
    return CC_ERR_OOM;
  } catch (const std::exception &e) {
    if (ctx) ctx->c.last_error = e.what();
    return CC_ERR_CUDA;
  }
}

}  // namespace

extern "C" {

int cc_set_default_allocator(void *(*alloc)(size_t, void *), void (*free_fn)(void *, void *),
                             void *user) {
  if ((alloc == nullptr) != (free_fn == nullptr)) return CC_ERR_ARG;
  std::lock_guard<std::mutex> lk(cdfns::g_mu);
  cdfns::g_default_alloc.alloc = alloc;
  cdfns::g_default_alloc.free = free_fn;
  cdfns::g_default_alloc.user = user;
  return CC_OK;
}

int cc_set_allocator(cc_ctx *ctx, void *(*alloc)(size_t, void *),
                     void (*free_fn)(void *, void *), void *user) {
  if (!ctx || (alloc == nullptr) != (free_fn == nullptr)) return CC_ERR_ARG;
  cdfns::Allocator &al = ctx->c.al;
  al.alloc = alloc;
  al.free = free_fn;
  al.user = user;
  return CC_OK;
}

int cc_set_default_stream(void *stream) {
  std::lock_guard<std::mutex> lk(cdfns::g_mu);
  cdfns::g_default_stream = static_cast<cudaStream_t>(stream);
  return CC_OK;
}

int cc_init_chunked(int n_occ, int n_virt, int n_aux, const double *eps, cc_ctx **out) {
  if (!out) return CC_ERR_ARG;
  *out = nullptr;
  cc_ctx *ctx = nullptr;
  try {
    ctx = new cc_ctx;
  } catch (...) {
    return CC_ERR_OOM;
  }
  {
    std::lock_guard<std::mutex> lk(cdfns::g_mu);
    ctx->c.al = cdfns::g_default_alloc;
    ctx->c.al.in_use = ctx->c.al.peak = ctx->c.al.window = ctx->c.al.limit = 0;
    ctx->c.st = cdfns::g_default_stream;
  }
  const int rc = guarded(ctx, [&] {
    ctx->c.create(n_occ, n_virt, n_aux, eps);
    return CC_OK;
  });
  if (rc != CC_OK) {
    delete ctx;
    return rc;
  }
  *out = ctx;
  return CC_OK;
}

int cc_add_cholesky(cc_ctx *ctx, int p0, int p1, const double *L_chunk) {
  if (!ctx) return CC_ERR_ARG;
  return guarded(ctx, [&] {
    ctx->c.add_chunk(p0, p1, L_chunk);
    return CC_OK;
  });
}

int cc_add_cholesky_dev(cc_ctx *ctx, int p0, int p1, const double *L_chunk_dev) {
  if (!ctx) return CC_ERR_ARG;
  return guarded(ctx, [&] {
    ctx->c.add_chunk(p0, p1, L_chunk_dev, true);
    return CC_OK;
  });
}

int cc_init(int n_occ, int n_virt, int n_aux, const double *eps, const double *L, cc_ctx **out) {
  if (!out) return CC_ERR_ARG;
  *out = nullptr;
  if (!L) return CC_ERR_ARG;
  cc_ctx *ctx = nullptr;
  int rc = cc_init_chunked(n_occ, n_virt, n_aux, eps, &ctx);
  if (rc != CC_OK) return rc;
  rc = guarded(ctx, [&] {
    ctx->c.add_chunk(0, n_aux, L);
    ctx->c.validate_input();
    return CC_OK;
  });
  if (rc != CC_OK) {
    delete ctx;
    return rc;
  }
  *out = ctx;
  return CC_OK;
}

int cc_set_precision(cc_ctx *ctx, int tier) {
  if (!ctx) return CC_ERR_ARG;
  if (tier < CC_TIER_FP64 || tier > CC_TIER_FP16X3) return CC_ERR_ARG;
  ctx->c.tier = tier;
  ctx->c.hbar_done = false;
  ctx->c.cc_done_tier = -1;  // an explicit choice also sets H-bar's tier
  return CC_OK;
}

int cc_set_precision_eom(cc_ctx *ctx, int tier) {
  if (!ctx) return CC_ERR_ARG;
  if (tier < -1 || tier > CC_TIER_FP16X3) return CC_ERR_ARG;
  ctx->c.eom_tier = tier;
  return CC_OK;
}

int cc_set_stream(cc_ctx *ctx, void *stream) {
  if (!ctx) return CC_ERR_ARG;
  ctx->c.st = static_cast<cudaStream_t>(stream);
  ctx->c.eng.st = ctx->c.st;
  return CC_OK;
}

int cc_set_slab_budget(cc_ctx *ctx, size_t bytes) {
  if (!ctx || bytes < 4096) return CC_ERR_ARG;
  ctx->c.slab_budget = bytes;
  return CC_OK;
}

int cc_get_sizes(const cc_ctx *ctx, int *n_occ, int *n_virt, int *n_aux) {
  if (!ctx) return CC_ERR_ARG;
  if (n_occ) *n_occ = ctx->c.o;
  if (n_virt) *n_virt = ctx->c.v;
  if (n_aux) *n_aux = ctx->c.X;
  return CC_OK;
}

int fns_truncate(cc_ctx *ctx, double threshold, int *n_virt_kept) {
  if (!ctx) return CC_ERR_ARG;
  if (!(threshold >= 0)) return CC_ERR_ARG;
  return guarded(ctx, [&] {
    const int rc = ctx->c.fns(threshold, -1);
    if (n_virt_kept) *n_virt_kept = ctx->c.v;
    return rc;
  });
}

int fns_truncate_count(cc_ctx *ctx, int n_keep) {
  if (!ctx || n_keep < 1) return CC_ERR_ARG;
  return guarded(ctx, [&] { return ctx->c.fns(0.0, n_keep); });
}

int fns_get_occupations(const cc_ctx *ctx, double *occ, int n) {
  if (!ctx || !occ) return CC_ERR_ARG;
  const auto &f = ctx->c.fns_occ;
  if (f.empty()) return CC_ERR_STATE;
  if (n < static_cast<int>(f.size())) return CC_ERR_ARG;
  std::memcpy(occ, f.data(), sizeof(double) * f.size());
  return CC_OK;
}

int ccsd_solve(cc_ctx *ctx, double tol, int max_iter, double *e_corr, int *n_iter) {
  if (!ctx || !e_corr) return CC_ERR_ARG;
  return guarded(ctx, [&] { return ctx->c.ccsd(tol, max_iter, e_corr, n_iter); });
}

int ipeom_solve(cc_ctx *ctx, int n_roots, double tol, int max_iter, double *omega, double *r1_weight,
                int *n_iter) {
  if (!ctx || !omega) return CC_ERR_ARG;
  return guarded(ctx, [&] {
    return ctx->c.ipeom(n_roots, tol, max_iter, omega, r1_weight, n_iter);
  });
}

int ipeom_solve_lr(cc_ctx *ctx, int n_roots, double tol, int max_iter, double *omega,
                   double *r_host, double *l_host, double *pole, int *n_iter) {
  if (!ctx || !omega || n_roots < 1) return CC_ERR_ARG;
  return guarded(ctx, [&] {
    Ctx &c = ctx->c;
    if (!c.ccsd_done) cdfns::fail(CC_ERR_STATE, "ipeom needs a converged ccsd_solve");
    if (n_roots > c.dim_ip() || n_roots > 64) cdfns::fail(CC_ERR_ARG, "n_roots out of range");
    const long dim = c.dim_ip();
    const size_t bytes = sizeof(cdfns::cplx) * n_roots * dim;
    cdfns::Buf R(&c.al, bytes), L(&c.al, bytes);
    const int rc = c.ipeom_lr(n_roots, tol, max_iter, omega, R.c(), L.c(), n_iter);
    if (r_host) CUDA_CHECK(cudaMemcpyAsync(r_host, R.p, bytes, cudaMemcpyDeviceToHost, c.st));
    if (l_host) CUDA_CHECK(cudaMemcpyAsync(l_host, L.p, bytes, cudaMemcpyDeviceToHost, c.st));
    if (pole) {
      // sum_i l^i r_i over the 1h block, per root
      std::vector<cdfns::cplx> r1(static_cast<size_t>(n_roots) * c.o), l1(r1.size());
      CUDA_CHECK(cudaMemcpy2DAsync(r1.data(), sizeof(cdfns::cplx) * c.o, R.p,
                                   sizeof(cdfns::cplx) * dim, sizeof(cdfns::cplx) * c.o, n_roots,
                                   cudaMemcpyDeviceToHost, c.st));
      CUDA_CHECK(cudaMemcpy2DAsync(l1.data(), sizeof(cdfns::cplx) * c.o, L.p,
                                   sizeof(cdfns::cplx) * dim, sizeof(cdfns::cplx) * c.o, n_roots,
                                   cudaMemcpyDeviceToHost, c.st));
      CUDA_CHECK(cudaStreamSynchronize(c.st));
      for (int k = 0; k < n_roots; ++k) {
        double re = 0, im = 0;
        for (int i = 0; i < c.o; ++i) {
          const cdfns::cplx a = l1[static_cast<size_t>(k) * c.o + i];
          const cdfns::cplx b = r1[static_cast<size_t>(k) * c.o + i];
          re += a.x * b.x - a.y * b.y;
          im += a.x * b.y + a.y * b.x;
        }
        pole[2 * k] = re;
        pole[2 * k + 1] = im;
      }
    }
    CUDA_CHECK(cudaStreamSynchronize(c.st));
    return rc;
  });
}

int cc_get_amplitudes(const cc_ctx *cctx, double *t1_host, double *t2_host) {
  cc_ctx *ctx = const_cast<cc_ctx *>(cctx);
  if (!ctx || !t1_host || !t2_host) return CC_ERR_ARG;
  return guarded(ctx, [&] {
    Ctx &c = ctx->c;
    if (!c.amps) cdfns::fail(CC_ERR_STATE, "no amplitudes yet");
    const long na = c.n_amp();
    cdfns::Buf vec(&c.al, sizeof(cdfns::cplx) * na);
    c.ensure_pairs();
    cdfns::pack_amps(c.t1.c(), c.t2.c(), c.o, c.v, c.ij_i.as<int>(), c.ij_j.as<int>(), c.ab_a.as<int>(),
                     c.ab_b.as<int>(), vec.c(), c.st);
    const long n1 = static_cast<long>(c.o) * c.v;
    CUDA_CHECK(cudaMemcpyAsync(t1_host, vec.p, sizeof(cdfns::cplx) * n1, cudaMemcpyDeviceToHost, c.st));
    CUDA_CHECK(cudaMemcpyAsync(t2_host, vec.c() + n1, sizeof(cdfns::cplx) * (na - n1),
                               cudaMemcpyDeviceToHost, c.st));
    CUDA_CHECK(cudaStreamSynchronize(c.st));
    return CC_OK;
  });
}

int cc_reset_amplitudes(cc_ctx *ctx) {
  if (!ctx) return CC_ERR_ARG;
  ctx->c.amps = false;
  ctx->c.amps_user = false;
  ctx->c.ccsd_done = false;
  ctx->c.hbar_done = false;
  return CC_OK;
}

int cc_set_amplitudes(cc_ctx *ctx, const double *t1_host, const double *t2_host) {
  if (!ctx || !t1_host || !t2_host) return CC_ERR_ARG;
  return guarded(ctx, [&] {
    Ctx &c = ctx->c;
    c.ensure_ready();
    const long na = c.n_amp();
    const long n1 = static_cast<long>(c.o) * c.v;
    cdfns::Buf vec(&c.al, sizeof(cdfns::cplx) * na);
    CUDA_CHECK(cudaMemcpyAsync(vec.p, t1_host, sizeof(cdfns::cplx) * n1, cudaMemcpyHostToDevice, c.st));
    CUDA_CHECK(cudaMemcpyAsync(vec.c() + n1, t2_host, sizeof(cdfns::cplx) * (na - n1),
                               cudaMemcpyHostToDevice, c.st));
    c.B(c.t1, n1);
    c.B(c.t2, static_cast<long>(c.o) * c.o * c.v * c.v);
    cdfns::unpack_amps(vec.c(), c.o, c.v, c.t1.c(), c.t2.c(), c.st);
    CUDA_CHECK(cudaStreamSynchronize(c.st));
    c.amps = true;
    c.amps_user = true;
    c.ccsd_done = false;
    c.hbar_done = false;
    return CC_OK;
  });
}

int cc_ladder_dev(cc_ctx *ctx, const double *tau_dev, double *out_dev) {
  if (!ctx || !tau_dev || !out_dev) return CC_ERR_ARG;
  return guarded(ctx, [&] {
    Ctx &c = ctx->c;
    c.ensure_ready();
    const size_t n = sizeof(cdfns::cplx) * c.o * c.o * c.v * c.v;
    CUDA_CHECK(cudaMemsetAsync(out_dev, 0, n, c.st));
    c.ladder(c.Lvv.c(), reinterpret_cast<const cdfns::cplx *>(tau_dev),
             reinterpret_cast<cdfns::cplx *>(out_dev), c.tier);
    CUDA_CHECK(cudaStreamSynchronize(c.st));
    c.settle_ladder_timing();
    c.eng.trace_flush();
    c.check_err_flag();
    return CC_OK;
  });
}

int cc_residual_dev(cc_ctx *ctx, const double *t1_dev, const double *t2_dev, double *r1_dev,
                    double *r2_dev) {
  if (!ctx || !t1_dev || !t2_dev || !r1_dev || !r2_dev) return CC_ERR_ARG;
  return guarded(ctx, [&] {
    Ctx &c = ctx->c;
    c.ensure_ready();
    c.residual(reinterpret_cast<const cdfns::cplx *>(t1_dev), reinterpret_cast<const cdfns::cplx *>(t2_dev),
               reinterpret_cast<cdfns::cplx *>(r1_dev), reinterpret_cast<cdfns::cplx *>(r2_dev));
    CUDA_CHECK(cudaStreamSynchronize(c.st));
    c.settle_ladder_timing();
    c.check_err_flag();
    return CC_OK;
  });
}

int ipeom_sigma_dev(cc_ctx *ctx, int n_vec, const double *r_dev, double *s_dev) {
  if (!ctx || !r_dev || !s_dev || n_vec < 1) return CC_ERR_ARG;
  return guarded(ctx, [&] {
    Ctx &c = ctx->c;
    if (!c.ccsd_done && !c.amps) cdfns::fail(CC_ERR_STATE, "sigma needs amplitudes");
    if (!c.hbar_done) c.build_hbar();
    c.sigma(n_vec, reinterpret_cast<const cdfns::cplx *>(r_dev), reinterpret_cast<cdfns::cplx *>(s_dev));
    CUDA_CHECK(cudaStreamSynchronize(c.st));
    c.check_err_flag();
    return CC_OK;
  });
}

int ipeom_left_sigma_dev(cc_ctx *ctx, int n_vec, const double *l_dev, double *s_dev) {
  if (!ctx || !l_dev || !s_dev || n_vec < 1) return CC_ERR_ARG;
  return guarded(ctx, [&] {
    Ctx &c = ctx->c;
    if (!c.ccsd_done && !c.amps) cdfns::fail(CC_ERR_STATE, "sigma needs amplitudes");
    if (!c.hbar_done) c.build_hbar();
    c.left_sigma(n_vec, reinterpret_cast<const cdfns::cplx *>(l_dev),
                 reinterpret_cast<cdfns::cplx *>(s_dev));
    CUDA_CHECK(cudaStreamSynchronize(c.st));
    c.check_err_flag();
    return CC_OK;
  });
}

int cc_zgemm_dev(int tier, long M, long N, long K, const double *A, const double *B, double *C) {
  if (tier < CC_TIER_FP64 || tier > CC_TIER_FP16X3 || M < 1 || N < 1 || K < 1 || !A || !B || !C)
    return CC_ERR_ARG;
  return guarded(nullptr, [&] {
    static cdfns::Allocator al;
    cdfns::Engine eng;
    eng.al = &al;
    eng.st = cdfns::g_default_stream;
    int dev = 0;
    CUDA_CHECK(cudaGetDevice(&dev));
    CUDA_CHECK(cudaDeviceGetAttribute(&eng.num_sms, cudaDevAttrMultiProcessorCount, dev));
    cdfns::Buf err(&al, 16);
    CUDA_CHECK(cudaMemsetAsync(err.p, 0, 16, eng.st));
    eng.err_flag = err.as<int>();
    eng.trace_init();
    using cdfns::T;
    eng.contract(cdfns::C1(), T(reinterpret_cast<const cdfns::cplx *>(A), "mk", {M, K}),
                 T(reinterpret_cast<const cdfns::cplx *>(B), "nk", {N, K}), cdfns::C0(),
                 T(reinterpret_cast<const cdfns::cplx *>(C), "mn", {M, N}), tier);
    int e = 0;
    CUDA_CHECK(cudaMemcpyAsync(&e, err.p, sizeof(int), cudaMemcpyDeviceToHost, eng.st));
    CUDA_CHECK(cudaStreamSynchronize(eng.st));
    if (e) cdfns::fail(CC_ERR_TIMEOUT, "bounded wait expired");
    return CC_OK;
  });
}

int cc_cholesky_dev(long N, int r, const double *B_dev, double tau, int max_vec, double *L_dev,
                    long *pivots_host, int *n_vec) {
  if (N < 1 || r < 1 || max_vec < 1 || !B_dev || !L_dev || !n_vec || !(tau >= 0.0))
    return CC_ERR_ARG;
  return guarded(nullptr, [&] {
    int dev = 0, sms = 0;
    CUDA_CHECK(cudaGetDevice(&dev));
    CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    *n_vec = cdfns::pivoted_cholesky(reinterpret_cast<const cdfns::cplx *>(B_dev), N, r, tau,
                                     max_vec, reinterpret_cast<cdfns::cplx *>(L_dev), pivots_host,
                                     &cdfns::g_default_alloc, cdfns::g_default_stream, sms);
    return CC_OK;
  });
}

int cc_selftest_conversions(const double *x_dev, long n, long long *mismatches) {
  if (!x_dev || n < 0 || !mismatches) return CC_ERR_ARG;
  return guarded(nullptr, [&] {
    cdfns::Buf bad(&cdfns::g_default_alloc, 2 * sizeof(unsigned long long));
    const cudaStream_t st = cdfns::noalloc_stream();
    cdfns::conversion_check(x_dev, n, bad.as<unsigned long long>(), st);
    unsigned long long h[2];
    CUDA_CHECK(cudaMemcpyAsync(h, bad.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaStreamSynchronize(st));
    mismatches[0] = static_cast<long long>(h[0]);
    mismatches[1] = static_cast<long long>(h[1]);
    return CC_OK;
  });
}

int cc_dump_integrals(cc_ctx *ctx, int block, double *out_host) {
  if (!ctx || !out_host || block < 0 || block > 3) return CC_ERR_ARG;
  return guarded(ctx, [&] {
    Ctx &c = ctx->c;
    c.ensure_ready();
    const long o = c.o, v = c.v, X = c.X;
    // strides: [P][p][q] blocks
    const cdfns::cplx *Loo = c.Loo.c(), *Lov = c.Lov.c(), *Lvo = c.Lvo.c(), *Lvv = c.Lvv.c();
    const long soo = o * o, sov = o * v, svv = v * v;
    int np, nq, nr, ns;
    cdfns::Buf out;
    // <pq||rs> = sum_P L_pr L_qs - L_ps L_qr
    switch (block) {
      case 0:  // <ij||kl>
        np = nq = nr = ns = c.o;
        out.reset(&c.al, sizeof(cdfns::cplx) * o * o * o * o);
        cdfns::dump_block(Loo, soo, o, 1, Loo, soo, o, 1, Loo, soo, o, 1, Loo, soo, o, 1, c.X, np, nq,
                          nr, ns, out.c(), c.st);
        break;
      case 1:  // <ij||ka>: L_ik L_ja - L_ia L_jk
        np = nq = nr = c.o;
        ns = c.v;
        out.reset(&c.al, sizeof(cdfns::cplx) * o * o * o * v);
        cdfns::dump_block(Loo, soo, o, 1, Lov, sov, v, 1, Lov, sov, v, 1, Loo, soo, o, 1, c.X, np, nq,
                          nr, ns, out.c(), c.st);
        break;
      case 2:  // <ij||ab>: L_ia L_jb - L_ib L_ja
        np = nq = c.o;
        nr = ns = c.v;
        out.reset(&c.al, sizeof(cdfns::cplx) * o * o * v * v);
        cdfns::dump_block(Lov, sov, v, 1, Lov, sov, v, 1, Lov, sov, v, 1, Lov, sov, v, 1, c.X, np, nq,
                          nr, ns, out.c(), c.st);
        break;
      default:  // <ia||bj>: L_ib L_aj - L_ij L_ab
        np = c.o;
        nq = c.v;
        nr = c.v;
        ns = c.o;
        out.reset(&c.al, sizeof(cdfns::cplx) * o * v * v * o);
        cdfns::dump_block(Lov, sov, v, 1, Lvo, sov, o, 1, Loo, soo, o, 1, Lvv, svv, v, 1, c.X, np, nq,
                          nr, ns, out.c(), c.st);
        break;
    }
    (void)X;
    CUDA_CHECK(cudaMemcpyAsync(out_host, out.p, out.bytes, cudaMemcpyDeviceToHost, c.st));
    CUDA_CHECK(cudaStreamSynchronize(c.st));
    return CC_OK;
  });
}

int cc_get_stats(const cc_ctx *ctx, double *out, int n) {
  if (!ctx || !out || n < 0 || n > 24) return CC_ERR_ARG;
  double s[24];
  std::memcpy(s, ctx->c.stat, sizeof(s));
  s[6] = static_cast<double>(cdfns::g_launches.load());
  s[11] = static_cast<double>(ctx->c.al.peak);
  s[12] = ctx->c.diis_depth;
  s[14] = static_cast<double>(ctx->c.al.in_use);
  std::memcpy(out, s, sizeof(double) * n);
  return CC_OK;
}

const char *cc_last_error(const cc_ctx *ctx) {
  if (ctx) return ctx->c.last_error.c_str();
  return cdfns::g_last_error.c_str();
}

void cc_free(cc_ctx *ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->c.st);
  cdfns::drop_graphs(&ctx->c);
  delete ctx;
}

int cc_set_graphs(cc_ctx *ctx, int on) {
  if (!ctx) return CC_ERR_ARG;
  ctx->c.use_graphs = on != 0;
  return CC_OK;
}

int cc_set_memory_limit(cc_ctx *ctx, size_t bytes) {
  if (!ctx) return CC_ERR_ARG;
  if (bytes && bytes < ctx->c.al.in_use) return CC_ERR_ARG;
  ctx->c.al.limit = bytes;
  return CC_OK;
}

int cc_batch_ipeom(cc_ctx **systems, int n_sys, int n_roots, double tol, int max_iter,
                   double *omega, double *r1_weight, int *n_iter, int *status) {
  if (!systems || n_sys < 1 || !omega || !status) return CC_ERR_ARG;
  for (int q = 0; q < n_sys; ++q)
    if (!systems[q]) return CC_ERR_ARG;
  for (int q = 0; q < n_sys; ++q)
    for (int r = q + 1; r < n_sys; ++r)
      if (systems[q] == systems[r]) return CC_ERR_ARG;
  if (!(tol > 0) || max_iter < 1 || n_roots < 1) return CC_ERR_ARG;
  return guarded(systems[0], [&] {
    std::vector<cdfns::Ctx *> sys;
    for (int q = 0; q < n_sys; ++q) sys.push_back(&systems[q]->c);
    cdfns::run_ipeom(sys, n_roots, tol, max_iter, omega, r1_weight, n_iter, status,
                     systems[0]->c.use_graphs, false, nullptr, true);
    for (int q = 0; q < n_sys; ++q)
      if (status[q] != CC_OK) return CC_ERR_NOT_CONVERGED;
    return CC_OK;
  });
}

int cc_batch_solve(cc_ctx **systems, int n_sys, int n_roots, double ccsd_tol, double eom_tol,
                   int max_iter, double *e_corr, double *omega, double *r1_weight,
                   int *status) {
  if (!systems || n_sys < 1 || !e_corr || !omega || !status) return CC_ERR_ARG;
  for (int q = 0; q < n_sys; ++q)
    if (!systems[q]) return CC_ERR_ARG;
  for (int q = 0; q < n_sys; ++q)
    for (int r = q + 1; r < n_sys; ++r)
      if (systems[q] == systems[r]) return CC_ERR_ARG;
  if (!(ccsd_tol > 0) || !(eom_tol > 0) || max_iter < 1 || n_roots < 1) return CC_ERR_ARG;
  // CCSD system by system: a system that fails keeps its own status and
  // leaves the others untouched
  std::vector<int> cc_status(n_sys, CC_OK);
  for (int q = 0; q < n_sys; ++q) {
    e_corr[2 * q] = e_corr[2 * q + 1] = 0.0;
    cc_status[q] = guarded(systems[q], [&] {
      return systems[q]->c.ccsd(ccsd_tol, max_iter, e_corr + 2 * q, nullptr);
    });
  }
  // the batched IP-EOM over the systems whose CCSD converged
  std::vector<cc_ctx *> ok;
  std::vector<int> idx;
  for (int q = 0; q < n_sys; ++q) {
    status[q] = cc_status[q];
    for (int r = 0; r < n_roots; ++r) {
      omega[2L * (static_cast<long>(q) * n_roots + r)] = 0.0;
      omega[2L * (static_cast<long>(q) * n_roots + r) + 1] = 0.0;
      if (r1_weight) r1_weight[static_cast<long>(q) * n_roots + r] = 0.0;
    }
    if (cc_status[q] == CC_OK) {
      ok.push_back(systems[q]);
      idx.push_back(q);
    }
  }
  if (!ok.empty()) {
    const int m = static_cast<int>(ok.size());
    std::vector<double> w(2L * m * n_roots), r1(static_cast<size_t>(m) * n_roots);
    std::vector<int> st(m);
    const int rc = cc_batch_ipeom(ok.data(), m, n_roots, eom_tol, max_iter, w.data(), r1.data(),
                                  nullptr, st.data());
    if (rc != CC_OK && rc != CC_ERR_NOT_CONVERGED) {
      for (int j = 0; j < m; ++j) status[idx[j]] = rc;
      if (ok[0] != systems[0]) systems[0]->c.last_error = ok[0]->c.last_error;
      return rc;
    }
    for (int j = 0; j < m; ++j) {
      const int q = idx[j];
      status[q] = st[j];
      for (int r = 0; r < n_roots; ++r) {
        omega[2L * (static_cast<long>(q) * n_roots + r)] = w[2L * (static_cast<long>(j) * n_roots + r)];
        omega[2L * (static_cast<long>(q) * n_roots + r) + 1] =
            w[2L * (static_cast<long>(j) * n_roots + r) + 1];
        if (r1_weight) r1_weight[static_cast<long>(q) * n_roots + r] = r1[static_cast<long>(j) * n_roots + r];
      }
    }
  }
  for (int q = 0; q < n_sys; ++q)
    if (status[q] != CC_OK) return CC_ERR_NOT_CONVERGED;
  return CC_OK;
}

int cc_begin_fns_stream(cc_ctx *ctx) {
  if (!ctx) return CC_ERR_ARG;
  return guarded(ctx, [&] {
    ctx->c.begin_fns_stream();
    return CC_OK;
  });
}

int fns_stream_truncate(cc_ctx *ctx, double threshold, int n_keep, int *n_virt_kept) {
  if (!ctx || (n_keep <= 0 && !(threshold >= 0))) return CC_ERR_ARG;
  return guarded(ctx, [&] {
    const int nk = ctx->c.fns_stream_truncate(threshold, n_keep);
    if (n_virt_kept) *n_virt_kept = nk;
    return CC_OK;
  });
}

int cc_set_wait_limit(unsigned long long ns) {
  cdfns::tc_set_wait_limit(ns);
  return CC_OK;
}

int cc_set_fault_injection(cc_ctx *ctx, int kind, int at_iteration) {
  if (!ctx || kind < 0 || kind > 2 || (kind && at_iteration < 1)) return CC_ERR_ARG;
  ctx->c.inject_kind = kind;
  ctx->c.inject_at = at_iteration;
  return CC_OK;
}

}  // extern "C"
