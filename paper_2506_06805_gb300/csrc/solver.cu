// Host orchestration of CD/FNS IP-EOM-CCSD on one GPU.
//
// Storage policy (the implementation section of the paper): integrals with
// at most two virtual indices are stored (<ij||kl>, <ij||ka>, <ij||ab>,
// <ia||bj>); everything with three or four virtual indices is formed from
// the Cholesky vectors (Eq. 23) inside the contraction that needs it.
#include <cusolverDn.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>

#include "solver.h"

namespace cdfns {

namespace {

double now_ms() {
  return std::chrono::duration<double, std::milli>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Solver {
  cusolverDnHandle_t h = nullptr;
  cusolverDnParams_t p = nullptr;
  ~Solver() {
    if (p) cusolverDnDestroyParams(p);
    if (h) cusolverDnDestroy(h);
  }
};

Solver &solver_for(cudaStream_t st) {
  thread_local Solver s;
  if (!s.h) {
    if (cusolverDnCreate(&s.h) != CUSOLVER_STATUS_SUCCESS) fail(CC_ERR_CUDA, "cusolverDnCreate failed");
    if (cusolverDnCreateParams(&s.p) != CUSOLVER_STATUS_SUCCESS)
      fail(CC_ERR_CUDA, "cusolverDnCreateParams failed");
  }
  cusolverDnSetStream(s.h, st);
  return s;
}

// Hermitian eigensolver on a column-major n x n matrix (in place: vectors).
void heevd(Allocator *al, cudaStream_t st, cplx *A, int n, double *w) {
  Solver &s = solver_for(st);
  int lwork = 0;
  if (cusolverDnZheevd_bufferSize(s.h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n,
                                  reinterpret_cast<cuDoubleComplex *>(A), n, w,
                                  &lwork) != CUSOLVER_STATUS_SUCCESS)
    fail(CC_ERR_CUDA, "zheevd buffer size failed");
  Buf work(al, sizeof(cuDoubleComplex) * std::max(lwork, 1));
  Buf info(al, sizeof(int));
  if (cusolverDnZheevd(s.h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n,
                       reinterpret_cast<cuDoubleComplex *>(A), n, w, work.as<cuDoubleComplex>(),
                       lwork, info.as<int>()) != CUSOLVER_STATUS_SUCCESS)
    fail(CC_ERR_CUDA, "zheevd failed");
  int hinfo = 0;
  CUDA_CHECK(cudaMemcpyAsync(&hinfo, info.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  CUDA_CHECK(cudaStreamSynchronize(st));
  if (hinfo != 0) fail(CC_ERR_NUMERIC, "zheevd info " + std::to_string(hinfo));
}

void h2d(void *dst, const void *src, size_t n, cudaStream_t st) {
  CUDA_CHECK(cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, st));
}
void d2h(void *dst, const void *src, size_t n, cudaStream_t st) {
  CUDA_CHECK(cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, st));
  CUDA_CHECK(cudaStreamSynchronize(st));
}
void d2d(void *dst, const void *src, size_t n, cudaStream_t st) {
  CUDA_CHECK(cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToDevice, st));
}
void zero(void *dst, size_t n, cudaStream_t st) { CUDA_CHECK(cudaMemsetAsync(dst, 0, n, st)); }

}  // namespace

// General complex eigensolver (right vectors) on a column-major m x m matrix.
void geev_dev(Allocator *al, cudaStream_t st, cplx *A, int m, cplx *w, cplx *vr) {
  Solver &s = solver_for(st);
  size_t dbytes = 0, hbytes = 0;
  if (cusolverDnXgeev_bufferSize(s.h, s.p, CUSOLVER_EIG_MODE_NOVECTOR, CUSOLVER_EIG_MODE_VECTOR, m,
                                 CUDA_C_64F, A, m, CUDA_C_64F, w, CUDA_C_64F, nullptr, m,
                                 CUDA_C_64F, vr, m, CUDA_C_64F, &dbytes,
                                 &hbytes) != CUSOLVER_STATUS_SUCCESS)
    fail(CC_ERR_CUDA, "Xgeev buffer size failed");
  Buf dwork(al, std::max<size_t>(dbytes, 16));
  std::vector<char> hwork(std::max<size_t>(hbytes, 16));
  Buf info(al, sizeof(int));
  if (cusolverDnXgeev(s.h, s.p, CUSOLVER_EIG_MODE_NOVECTOR, CUSOLVER_EIG_MODE_VECTOR, m, CUDA_C_64F, A,
                      m, CUDA_C_64F, w, CUDA_C_64F, nullptr, m, CUDA_C_64F, vr, m, CUDA_C_64F,
                      dwork.p, dbytes, hwork.data(), hbytes,
                      info.as<int>()) != CUSOLVER_STATUS_SUCCESS)
    fail(CC_ERR_CUDA, "Xgeev failed");
  int hinfo = 0;
  CUDA_CHECK(cudaMemcpyAsync(&hinfo, info.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  CUDA_CHECK(cudaStreamSynchronize(st));
  if (hinfo != 0) fail(CC_ERR_NUMERIC, "Xgeev info " + std::to_string(hinfo));
}


// ===========================================================================
// lifecycle
// ===========================================================================
void Ctx::create(int n_occ, int n_virt, int n_aux, const double *eps_host) {
  if (n_occ < 1 || n_virt < 1 || n_aux < 1) fail(CC_ERR_ARG, "n_occ, n_virt, n_aux must be >= 1");
  if (!eps_host) fail(CC_ERR_ARG, "eps is NULL");
  o = n_occ;
  v = n_virt;
  X = n_aux;
  v_input = v;
  eps.assign(eps_host, eps_host + o + v);
  for (double e : eps)
    if (!std::isfinite(e)) fail(CC_ERR_INPUT, "eps contains NaN or Inf");
  int dev = 0;
  CUDA_CHECK(cudaGetDevice(&dev));
  CUDA_CHECK(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
  eng.al = &al;
  eng.st = st;
  eng.num_sms = num_sms;
  eng.trace_init();
  err_d.reset(&al, 64);
  stats_d.reset(&al, 64);
  red.reset(&al, 4096 * sizeof(cplx));
  zero(err_d.p, 64, st);
  zero(stats_d.p, 64, st);
  eng.err_flag = err_d.as<int>();
  eps_d.reset(&al, sizeof(double) * (o + v));
  h2d(eps_d.p, eps.data(), sizeof(double) * (o + v), st);
  const size_t cs = sizeof(cplx);
  Loo.reset(&al, cs * X * o * o);
  Lov.reset(&al, cs * X * o * v);
  Lvo.reset(&al, cs * X * v * o);
  Lvv.reset(&al, cs * X * v * v);
  have_P.assign(X, 0);
  n_have = 0;
}

void Ctx::add_chunk(int p0, int p1, const double *L, bool on_device) {
  if (p0 < 0 || p1 > X || p0 >= p1) fail(CC_ERR_ARG, "cholesky chunk range");
  if (!L) fail(CC_ERR_ARG, "L chunk is NULL");
  if (fns_stream == 2) {
    rotate_chunk(p0, p1, L, on_device);
    return;
  }
  if (ints || fns_stream == 3) fail(CC_ERR_STATE, "Cholesky vectors already consumed");
  const int n = o + v;
  const size_t per = sizeof(cplx) * n * n;
  if (on_device) {
    split_cholesky(reinterpret_cast<const cplx *>(L), p1 - p0, p0, o, v, Loo.c(), Lov.c(), Lvo.c(),
                   fns_stream == 1 ? nullptr : Lvv.c(), stats_d.as<unsigned long long>(), st);
  } else {
    const int step = static_cast<int>(std::max<size_t>(1, (size_t(256) << 20) / per));
    Buf stage(&al, per * std::min(step, p1 - p0));
    for (int q0 = p0; q0 < p1; q0 += step) {
      const int q1 = std::min(p1, q0 + step);
      h2d(stage.p, L + static_cast<size_t>(q0 - p0) * 2 * n * n, per * (q1 - q0), st);
      split_cholesky(stage.c(), q1 - q0, q0, o, v, Loo.c(), Lov.c(), Lvo.c(),
                     fns_stream == 1 ? nullptr : Lvv.c(), stats_d.as<unsigned long long>(), st);
    }
  }
  CUDA_CHECK(cudaStreamSynchronize(st));
  for (int P = p0; P < p1; ++P)
    if (!have_P[P]) {
      have_P[P] = 1;
      ++n_have;
    }
}

void Ctx::validate_input() {
  if (n_have < X) fail(CC_ERR_STATE, "not every Cholesky vector has been given");
  if (input_checked) return;
  unsigned long long s[3];
  d2h(s, stats_d.p, sizeof(s), st);
  double mx, asym;
  std::memcpy(&mx, &s[0], 8);
  std::memcpy(&asym, &s[1], 8);
  if (s[2] != 0) fail(CC_ERR_INPUT, "L contains NaN or Inf");
  if (asym > 1e-12 * std::max(mx, 1e-300))
    fail(CC_ERR_INPUT, "L^P is not Hermitian (max |L_pq - conj(L_qp)| = " + std::to_string(asym) + ")");
  input_checked = true;
}

// Integrals are built at the first solver call, in the tier current then.
void Ctx::ensure_ready() {
  if (fns_stream == 1 || fns_stream == 2)
    fail(CC_ERR_STATE, "streamed natural spinors: both passes over the Cholesky vectors must end first");
  validate_input();
  if (!ints) build_integrals();
}

void Ctx::settle_sigma_timing() {
  for (const auto &t : sig_timing) {
    CUDA_CHECK(cudaEventSynchronize(t->e1));
    float ms = 0;
    CUDA_CHECK(cudaEventElapsedTime(&ms, t->e0, t->e1));
    stat[16] += ms;
    stat[17] += 1;
  }
  sig_timing.clear();
}

void Ctx::maybe_inject(int kind, int iteration, cplx *target) {
  if (inject_kind != kind || inject_at != iteration) return;
  const cplx bad = mk(std::nan(""), 0.0);
  h2d(target, &bad, sizeof(cplx), st);
  CUDA_CHECK(cudaStreamSynchronize(st));
  inject_kind = 0;
}

void Ctx::check_err_flag() {
  int e = 0;
  d2h(&e, err_d.p, sizeof(int), st);
  if (e) {
    zero(err_d.p, sizeof(int), st);
    fail(CC_ERR_TIMEOUT, "a bounded device wait expired in a tensor-core kernel");
  }
}

void Ctx::ensure_pairs() {
  if (pairs_o == o && pairs_v == v) return;
  ij_i.reset(&al, sizeof(int) * std::max<long>(nij(), 1));
  ij_j.reset(&al, sizeof(int) * std::max<long>(nij(), 1));
  ab_a.reset(&al, sizeof(int) * std::max<long>(nab(), 1));
  ab_b.reset(&al, sizeof(int) * std::max<long>(nab(), 1));
  make_pairs(o, ij_i.as<int>(), ij_j.as<int>(), st);
  make_pairs(v, ab_a.as<int>(), ab_b.as<int>(), st);
  pairs_o = o;
  pairs_v = v;
}

// <pq||rs> = sum_P (L_pr L_qs - L_ps L_qr)  (Eq. 23), stored blocks only.
void Ctx::build_integrals() {
  const int tr = int_tier();
  const long oo = static_cast<long>(o) * o, ov = static_cast<long>(o) * v;
  B(oooo, oo * oo);
  B(ooov, oo * ov);
  B(oovv, oo * v * v);
  B(ovvo, ov * v * o);
  Buf tmp(&al, sizeof(cplx) * std::max(oo * oo, oo * v * v));
  // <mn||ij>
  eng.contract(C1(), T(Loo.c(), "Pmi", {X, o, o}), T(Loo.c(), "Pnj", {X, o, o}), C0(),
               T(tmp.c(), "mnij", {o, o, o, o}), tr);
  eng.permute_into(C1(), T(tmp.c(), "mnij", {o, o, o, o}), C0(), T(oooo.c(), "mnij", {o, o, o, o}));
  eng.permute_into(Cr(-1), T(tmp.c(), "mnji", {o, o, o, o}), C1(), T(oooo.c(), "mnij", {o, o, o, o}));
  // <mn||ie>
  eng.contract(C1(), T(Loo.c(), "Pmi", {X, o, o}), T(Lov.c(), "Pne", {X, o, v}), C0(),
               T(ooov.c(), "mnie", {o, o, o, v}), tr);
  eng.contract(Cr(-1), T(Lov.c(), "Pme", {X, o, v}), T(Loo.c(), "Pni", {X, o, o}), C1(),
               T(ooov.c(), "mnie", {o, o, o, v}), tr);
  // <ij||ab>
  eng.contract(C1(), T(Lov.c(), "Pia", {X, o, v}), T(Lov.c(), "Pjb", {X, o, v}), C0(),
               T(tmp.c(), "ijab", {o, o, v, v}), tr);
  eng.permute_into(C1(), T(tmp.c(), "ijab", {o, o, v, v}), C0(), T(oovv.c(), "ijab", {o, o, v, v}));
  eng.permute_into(Cr(-1), T(tmp.c(), "ijba", {o, o, v, v}), C1(), T(oovv.c(), "ijab", {o, o, v, v}));
  // <mb||ej>
  eng.contract(C1(), T(Lov.c(), "Pme", {X, o, v}), T(Lvo.c(), "Pbj", {X, v, o}), C0(),
               T(ovvo.c(), "mbej", {o, v, v, o}), tr);
  eng.contract(Cr(-1), T(Loo.c(), "Pmj", {X, o, o}), T(Lvv.c(), "Pbe", {X, v, v}), C1(),
               T(ovvo.c(), "mbej", {o, v, v, o}), tr);
  CUDA_CHECK(cudaStreamSynchronize(st));
  check_err_flag();
  eng.clear_pack_cache();
  ints = true;
}

cplx Ctx::energy(const cplx *t1p, const cplx *t2p) {
  // Eq. 15 with f_ia = 0: 1/4 <ij||ab> t_ij^ab + 1/2 <ij||ab> t_i^a t_j^b
  const long n2 = static_cast<long>(o) * o * v * v;
  Buf tmp(&al, sizeof(cplx) * o * v);
  eng.contract(C1(), T(oovv.c(), "ijab", {o, o, v, v}), T(t1p, "jb", {o, v}), C0(),
               T(tmp.c(), "ia", {o, v}), TIER_FP64);
  cplx* r = red.c();
  dot_dev(oovv.c(), t2p, n2, false, r + 2048, st, r);
  dot_dev(tmp.c(), t1p, static_cast<long>(o) * v, false, r + 2049, st, r + 1024);
  cplx h[2];
  d2h(h, r + 2048, sizeof(h), st);
  return mk(0.25 * h[0].x + 0.5 * h[1].x, 0.25 * h[0].y + 0.5 * h[1].y);
}

// ===========================================================================
// frozen natural spinors (Eqs. 24-28)
// ===========================================================================
int Ctx::fns(double threshold, int n_keep) {
  if (fns_stream) fail(CC_ERR_STATE, "use fns_stream_truncate with cc_begin_fns_stream");
  ensure_ready();
  if (ccsd_done || amps_user) fail(CC_ERR_STATE, "fns_truncate must precede ccsd_solve");
  const double t0 = now_ms();
  const long oo = static_cast<long>(o) * o;
  const int tr = TIER_FP64;
  // MP2 amplitudes t_ij^ab = <ab||ij> / D
  Buf tm1(&al, sizeof(cplx) * o * v), tm2(&al, sizeof(cplx) * oo * v * v);
  mp2_amplitudes(oovv.c(), eps_d.as<double>(), o, v, tm1.c(), tm2.c(), st);
  // Eq. 24: D_ab = 1/2 sum_ijc t_ij^ac conj(t_ij^bc); stored column-major
  Buf Dm(&al, sizeof(cplx) * v * v);
  // the o^2 v^3 density GEMM runs in the 3-product split tier when a
  // tensor-core tier is selected (relative error ~1e-6, far below the
  // spacing of occupations near any threshold)
  eng.contract(Cr(0.5), T(tm2.c(), "ijac", {o, o, v, v}), conj(T(tm2.c(), "ijbc", {o, o, v, v})),
               C0(), T(Dm.c(), "ba", {v, v}), int_tier());
  tm2.release();
  // Eq. 25
  Buf w(&al, sizeof(double) * v);
  heevd(&al, st, Dm.c(), v, w.as<double>());
  std::vector<double> occ(v);
  d2h(occ.data(), w.p, sizeof(double) * v, st);
  std::reverse(occ.begin(), occ.end());  // descending
  fns_occ = occ;
  int nk = n_keep;
  if (nk < 0) {
    nk = 0;
    for (double x : occ)
      if (x >= threshold) ++nk;
  }
  if (nk < 1) fail(CC_ERR_STATE, "FNS threshold keeps no virtual spinor");
  if (nk > v) fail(CC_ERR_ARG, "n_keep exceeds n_virt");
  // V~ rows: Vt[k][a] = eigenvector of the k-th largest occupation
  Buf Vt(&al, sizeof(cplx) * nk * v);
  eng.permute_into(C1(), Tv(Dm.c() + static_cast<long>(v - 1) * v, "ka", {nk, v}, {-v, 1}), C0(),
                   T(Vt.c(), "ka", {nk, v}));
  // Eq. 26: F^NS = V~^H diag(eps_v) V~  (column-major for the eigensolver)
  std::vector<cplx> Ed(static_cast<size_t>(v) * v, mk(0, 0));
  for (int a = 0; a < v; ++a) Ed[static_cast<size_t>(a) * v + a] = mk(eps[o + a], 0);
  Buf Ev(&al, sizeof(cplx) * v * v);
  h2d(Ev.p, Ed.data(), sizeof(cplx) * v * v, st);
  Buf EVt(&al, sizeof(cplx) * nk * v), Fm(&al, sizeof(cplx) * nk * nk);
  eng.contract(C1(), T(Vt.c(), "kb", {nk, v}), T(Ev.c(), "ab", {v, v}), C0(),
               T(EVt.c(), "ka", {nk, v}), tr);
  eng.contract(C1(), conj(T(Vt.c(), "ka", {nk, v})), T(EVt.c(), "la", {nk, v}), C0(),
               T(Fm.c(), "lk", {nk, nk}), tr);
  // Eq. 27
  Buf w2(&al, sizeof(double) * nk);
  heevd(&al, st, Fm.c(), nk, w2.as<double>());
  std::vector<double> ev(nk);
  d2h(ev.data(), w2.p, sizeof(double) * nk, st);
  // Eq. 28 (read as U = V~ Z~): U[a][l] = sum_k V~(a,k) Z(k,l)
  Buf U(&al, sizeof(cplx) * v * nk);
  eng.contract(C1(), T(Vt.c(), "ka", {nk, v}), T(Fm.c(), "lk", {nk, nk}), C0(),
               T(U.c(), "al", {v, nk}), tr);
  // rotate the virtual indices of L (Eq. 22 form)
  const int rt = int_tier();
  Buf Lov2(&al, sizeof(cplx) * X * o * nk), Lvo2(&al, sizeof(cplx) * X * nk * o);
  Buf Lvv2(&al, sizeof(cplx) * X * nk * nk);
  eng.contract(C1(), T(Lov.c(), "Pia", {X, o, v}), T(U.c(), "al", {v, nk}), C0(),
               T(Lov2.c(), "Pil", {X, o, nk}), rt);
  eng.contract(C1(), conj(T(U.c(), "al", {v, nk})), T(Lvo.c(), "Pai", {X, v, o}), C0(),
               T(Lvo2.c(), "Pli", {X, nk, o}), rt);
  {
    Buf tmp(&al, sizeof(cplx) * X * v * nk);
    eng.contract(C1(), T(Lvv.c(), "Pab", {X, v, v}), T(U.c(), "bl", {v, nk}), C0(),
                 T(tmp.c(), "Pal", {X, v, nk}), rt);
    eng.contract(C1(), conj(T(U.c(), "ak", {v, nk})), T(tmp.c(), "Pal", {X, v, nk}), C0(),
                 T(Lvv2.c(), "Pkl", {X, nk, nk}), rt);
  }
  CUDA_CHECK(cudaStreamSynchronize(st));
  check_err_flag();
  Lov = std::move(Lov2);
  Lvo = std::move(Lvo2);
  Lvv = std::move(Lvv2);
  v = nk;
  eps.resize(o + v);
  for (int a = 0; a < v; ++a) eps[o + a] = ev[a];
  eps_d.reset(&al, sizeof(double) * (o + v));
  h2d(eps_d.p, eps.data(), sizeof(double) * (o + v), st);
  ints = false;
  hbar_done = false;
  amps = false;
  eng.clear_cache();
  build_integrals();
  fns_done = true;
  stat[3] += now_ms() - t0;
  return CC_OK;
}

// ===========================================================================
// Streamed frozen natural spinors (Eqs. 24-28) for systems whose L_vv does
// not fit on the device (X v^2 complex: 184 GB at v = 1698, X = 4000). The
// first pass over the Cholesky chunks keeps only L_oo, L_ov and L_vo; the
// density of Eq. 24 is then built from MP2 amplitudes of one occupied index
// i at a time, D = sum_{i<j} T_ij T_ij^H with T_ij[a][c] = <ac||ij> / D_ij^ac
// (the unrestricted sum of Eq. 24 counts each pair twice with its 1/2), so
// the o^2 v^2 amplitudes are never held whole; U follows as in fns(). The
// second pass rotates each chunk's L_vv^P into the kept basis (U^H L^P U) as
// it arrives.
// ===========================================================================
void Ctx::begin_fns_stream() {
  if (n_have > 0 || ints || fns_stream) fail(CC_ERR_STATE, "cc_begin_fns_stream must precede cc_add_cholesky");
  if (ccsd_done || amps_user || fns_done) fail(CC_ERR_STATE, "natural spinors must precede CCSD");
  Lvv.release();
  fns_stream = 1;
}

int Ctx::fns_stream_truncate(double threshold, int n_keep) {
  if (fns_stream != 1) fail(CC_ERR_STATE, "fns_stream_truncate follows the first pass over the chunks");
  validate_input();
  const double t0 = now_ms();
  const int tr = int_tier();
  const long vv = static_cast<long>(v) * v;
  Buf Dm(&al, sizeof(cplx) * vv);
  zero(Dm.p, sizeof(cplx) * vv, st);
  {
    const long nmax = std::max(o - 1, 1);
    Buf G(&al, sizeof(cplx) * nmax * vv), tm(&al, sizeof(cplx) * nmax * vv);
    for (int i = 0; i + 1 < o; ++i) {
      const int nj = o - i - 1;
      // G[j'][a][b] = sum_P L^P_ai L^P_bj, j = i + 1 + j'
      eng.contract(C1(), Tv(Lvo.c() + i, "Pa", {X, v}, {static_cast<long>(v) * o, o}),
                   Tv(Lvo.c() + i + 1, "Pbj", {X, v, nj}, {static_cast<long>(v) * o, o, 1}), C0(),
                   T(G.c(), "jab", {nj, v, v}), tr);
      mp2_pair_amplitudes(G.c(), eps_d.as<double>(), o, v, i, nj, tm.c(), st);
      // D_ab += sum_{j,c} t_ij^ac conj(t_ij^bc), stored column-major
      eng.contract(C1(), T(tm.c(), "jac", {nj, v, v}), conj(T(tm.c(), "jbc", {nj, v, v})), C1(),
                   T(Dm.c(), "ba", {v, v}), tr);
    }
  }
  // Eq. 25
  Buf w(&al, sizeof(double) * v);
  heevd(&al, st, Dm.c(), v, w.as<double>());
  std::vector<double> occ(v);
  d2h(occ.data(), w.p, sizeof(double) * v, st);
  std::reverse(occ.begin(), occ.end());
  fns_occ = occ;
  int nk = n_keep;
  if (nk <= 0) {
    nk = 0;
    for (double x : occ)
      if (x >= threshold) ++nk;
  }
  if (nk < 1) fail(CC_ERR_STATE, "FNS threshold keeps no virtual spinor");
  if (nk > v) fail(CC_ERR_ARG, "n_keep exceeds n_virt");
  Buf Vt(&al, sizeof(cplx) * nk * v);
  eng.permute_into(C1(), Tv(Dm.c() + static_cast<long>(v - 1) * v, "ka", {nk, v}, {-v, 1}), C0(),
                   T(Vt.c(), "ka", {nk, v}));
  // Eqs. 26-28 in FP64, as in fns()
  std::vector<cplx> Ed(static_cast<size_t>(vv), mk(0, 0));
  for (int a = 0; a < v; ++a) Ed[static_cast<size_t>(a) * v + a] = mk(eps[o + a], 0);
  Buf Ev(&al, sizeof(cplx) * vv);
  h2d(Ev.p, Ed.data(), sizeof(cplx) * vv, st);
  Buf EVt(&al, sizeof(cplx) * nk * v), Fm(&al, sizeof(cplx) * nk * nk);
  eng.contract(C1(), T(Vt.c(), "kb", {nk, v}), T(Ev.c(), "ab", {v, v}), C0(),
               T(EVt.c(), "ka", {nk, v}), TIER_FP64);
  eng.contract(C1(), conj(T(Vt.c(), "ka", {nk, v})), T(EVt.c(), "la", {nk, v}), C0(),
               T(Fm.c(), "lk", {nk, nk}), TIER_FP64);
  Buf w2(&al, sizeof(double) * nk);
  heevd(&al, st, Fm.c(), nk, w2.as<double>());
  eps_kept.resize(nk);
  d2h(eps_kept.data(), w2.p, sizeof(double) * nk, st);
  U_fns.reset(&al, sizeof(cplx) * v * nk);
  eng.contract(C1(), T(Vt.c(), "ka", {nk, v}), T(Fm.c(), "lk", {nk, nk}), C0(),
               T(U_fns.c(), "al", {v, nk}), TIER_FP64);
  Lvv_kept.reset(&al, sizeof(cplx) * X * nk * nk);
  have_P2.assign(X, 0);
  n_have2 = 0;
  fns_stream = 2;
  CUDA_CHECK(cudaStreamSynchronize(st));
  check_err_flag();
  fns_ms = now_ms() - t0;
  return nk;
}

void Ctx::rotate_chunk(int p0, int p1, const double *L, bool on_device) {
  const double t0 = now_ms();
  const int n = o + v;
  const int nk = static_cast<int>(eps_kept.size());
  const int rt = int_tier();
  const size_t per = sizeof(cplx) * n * n;
  const int step = static_cast<int>(std::max<size_t>(1, (size_t(512) << 20) / per));
  const int cap = std::min(step, p1 - p0);
  Buf stage, lvv(&al, sizeof(cplx) * cap * v * v), tmp(&al, sizeof(cplx) * cap * v * nk);
  if (!on_device) stage.reset(&al, per * cap);
  Buf scratch_stats(&al, 64);
  zero(scratch_stats.p, 64, st);
  for (int q0 = p0; q0 < p1; q0 += step) {
    const int q1 = std::min(p1, q0 + step), nq = q1 - q0;
    const cplx *src = reinterpret_cast<const cplx *>(L) + static_cast<size_t>(q0 - p0) * n * n;
    if (!on_device) {
      h2d(stage.p, src, per * nq, st);
      src = stage.c();
    }
    split_cholesky(src, nq, 0, o, v, nullptr, nullptr, nullptr, lvv.c(),
                   scratch_stats.as<unsigned long long>(), st);
    eng.contract(C1(), T(lvv.c(), "Pab", {nq, v, v}), T(U_fns.c(), "bl", {v, nk}), C0(),
                 T(tmp.c(), "Pal", {nq, v, nk}), rt);
    eng.contract(C1(), conj(T(U_fns.c(), "ak", {v, nk})), T(tmp.c(), "Pal", {nq, v, nk}), C0(),
                 T(Lvv_kept.c() + static_cast<long>(q0) * nk * nk, "Pkl", {nq, nk, nk}), rt);
  }
  CUDA_CHECK(cudaStreamSynchronize(st));
  check_err_flag();
  for (int P = p0; P < p1; ++P)
    if (!have_P2[P]) {
      have_P2[P] = 1;
      ++n_have2;
    }
  fns_ms += now_ms() - t0;
  if (n_have2 == X) finish_fns_stream();
}

void Ctx::finish_fns_stream() {
  const int nk = static_cast<int>(eps_kept.size());
  const int rt = int_tier();
  Buf Lov2(&al, sizeof(cplx) * X * o * nk), Lvo2(&al, sizeof(cplx) * X * nk * o);
  eng.contract(C1(), T(Lov.c(), "Pia", {X, o, v}), T(U_fns.c(), "al", {v, nk}), C0(),
               T(Lov2.c(), "Pil", {X, o, nk}), rt);
  eng.contract(C1(), conj(T(U_fns.c(), "al", {v, nk})), T(Lvo.c(), "Pai", {X, v, o}), C0(),
               T(Lvo2.c(), "Pli", {X, nk, o}), rt);
  CUDA_CHECK(cudaStreamSynchronize(st));
  check_err_flag();
  Lov = std::move(Lov2);
  Lvo = std::move(Lvo2);
  Lvv = std::move(Lvv_kept);
  U_fns.release();
  v = nk;
  eps.resize(o + v);
  for (int a = 0; a < v; ++a) eps[o + a] = eps_kept[a];
  eps_d.reset(&al, sizeof(double) * (o + v));
  h2d(eps_d.p, eps.data(), sizeof(double) * (o + v), st);
  ints = false;
  hbar_done = false;
  amps = false;
  eng.clear_cache();
  fns_done = true;
  fns_stream = 3;
  stat[3] += fns_ms;
}

// ===========================================================================
// ladder: R2 += 1/2 sum_cd <ab||cd> tau_ij^cd with <ab||cd> from Lv (Eq. 23)
// ===========================================================================
void Ctx::ladder(const cplx *Lv, const cplx *tau, cplx *R2, int tr, const float *tau_amax) {
  ensure_pairs();
  const long vv = static_cast<long>(v) * v;
  const long n_ij = nij(), n_cd = nab(), n_ab = nab();
  if (n_ij == 0 || n_ab == 0) return;
  auto tm = std::make_shared<EventPair>();
  CUDA_CHECK(cudaEventCreate(&tm->e0));
  CUDA_CHECK(cudaEventCreate(&tm->e1));
  CUDA_CHECK(cudaEventRecord(tm->e0, st));
  Buf Rp(&al, sizeof(cplx) * n_ij * n_ab);
  // tau gather tables: row (i<j) -> (i*o + j)*vv, col (c<d) -> c*v + d
  std::vector<long> rows(n_ij), cols(n_cd);
  {
    long q = 0;
    for (int i = 0; i < o; ++i)
      for (int j = i + 1; j < o; ++j) rows[q++] = (static_cast<long>(i) * o + j) * vv;
    q = 0;
    for (int c = 0; c < v; ++c)
      for (int d = c + 1; d < v; ++d) cols[q++] = static_cast<long>(c) * v + d;
  }
  Buf rt(&al, sizeof(long) * n_ij), kt(&al, sizeof(long) * n_cd);
  h2d(rt.p, rows.data(), sizeof(long) * n_ij, st);
  h2d(kt.p, cols.data(), sizeof(long) * n_cd, st);
  const long Pstride[1] = {vv};
  const long Xd[1] = {X};
  const long *ptab = eng.table(std::vector<long>(Xd, Xd + 1), std::vector<long>(Pstride, Pstride + 1));
  const bool fast = tr != TIER_FP64;
  const size_t eb = fast ? tc_elem_bytes(tr) : sizeof(cplx);
  const size_t veb = fast ? sizeof(float2) : sizeof(cplx);

  if (!fast) {
    // K-major copy of L: LT[(a,c)][P]
    Buf LT(&al, sizeof(cplx) * vv * X);
    eng.permute_into(C1(), T(Lv, "Pac", {X, v, v}), C0(), T(LT.c(), "acP", {v, v, X}));
    long a0 = 0;
    Buf Vs, W;
    while (a0 < v - 1) {
      const long per_a = static_cast<long>(v) * (v - a0) * v;
      long nA = std::max<long>(1, static_cast<long>(slab_budget / (per_a * veb)));
      nA = std::min<long>(nA, v - 1 - a0);
      const long a1 = a0 + nA;
      const long p0 = a0 * v - a0 * (a0 + 1) / 2;
      const long p1 = a1 * v - a1 * (a1 + 1) / 2;
      const long np = p1 - p0;
      B(Vs, nA * per_a);
      B(W, np * n_cd);
      GemmDesc g1;
      g1.M = nA * v; g1.N = (v - a0) * v; g1.K = X;
      g1.A = LT.c() + a0 * v * X; g1.lda = X;
      g1.B = LT.c() + a0 * v * X; g1.ldb = X;
      g1.C = Vs.c(); g1.ldc = (v - a0) * v;
      gemm_f64(g1, st, num_sms);
      ladder_antisym(Vs.p, false, v, static_cast<int>(a0), static_cast<int>(nA), p0, p1,
                     ab_a.as<int>(), ab_b.as<int>(), ab_a.as<int>(), ab_b.as<int>(), TIER_FP64,
                     nullptr, nullptr, 0, W.c(), st);
      GemmDesc g2;
      g2.M = n_ij; g2.N = np; g2.K = n_cd;
      g2.A = tau; g2.am = rt.as<long>(); g2.ak = kt.as<long>();
      g2.B = W.c(); g2.ldb = n_cd;
      g2.C = Rp.c() + p0; g2.ldc = n_ab;
      gemm_f64(g2, st, num_sms);
      a0 = a1;
    }
  } else {
    const int kal = tc_k_align(tr);
    const long Kp1 = ((2L * X + kal - 1) / kal) * kal;
    const long Kp2 = ((2L * n_cd + kal - 1) / kal) * kal;
    const bool split = tier_split(tr);
    const bool f16 = tier_scaled(tr);
    Buf A1h(&al, eb * 2 * vv * Kp1), B1h(&al, eb * vv * Kp1), A2h(&al, eb * 2 * n_ij * Kp2);
    Buf A1l, B1l, A2l;
    if (split) {
      A1l.reset(&al, eb * 2 * vv * Kp1);
      B1l.reset(&al, eb * vv * Kp1);
      A2l.reset(&al, eb * 2 * n_ij * Kp2);
    }
    // FP16: operand maxima of L~ and tau, and a bound on |W|
    Buf amx(&al, 4 * sizeof(float));
    float *amx_L = f16 ? amx.as<float>() : nullptr;
    // tau's maximum over i<j, c<d is its maximum over all elements (the
    // others are zero or equal in magnitude by antisymmetry), so a caller's
    // whole-tensor maximum serves
    const float *amx_t = f16 ? (tau_amax ? tau_amax : amx.as<float>() + 1) : nullptr;
    float *amx_W = f16 ? amx.as<float>() + 2 : nullptr;
    {
      Engine::Region r = eng.region("ladder pack");
      if (f16) {
        tc_absmax(Lv, nullptr, ptab, 1, vv, X, amx_L, st);
        if (!tau_amax)
          tc_absmax(tau, rt.as<long>(), kt.as<long>(), 0, n_ij, n_cd, amx.as<float>() + 1, st);
        // |W| <= 2 max |V|: each GEMM1 raises amx_W to twice the largest
        // slab value it writes, before the antisymmetriser of its block
        zero(amx_W, sizeof(float), st);
      }
      tc_pack_A(Lv, nullptr, ptab, 1, false, vv, X, Kp1, tr, A1h.p, A1l.p, st, amx_L);
      tc_pack_B(Lv, nullptr, ptab, 1, false, vv, X, Kp1, tr, B1h.p, B1l.p, st, amx_L);
      tc_pack_A(tau, rt.as<long>(), kt.as<long>(), 0, false, n_ij, n_cd, Kp2, tr, A2h.p, A2l.p,
                st, amx_t);
    }
    long a0 = 0;
    Buf Vs, Wh, Wl;
    auto off = [&](const Buf &b, long elems) -> const void * {
      return b.p ? static_cast<const void *>(static_cast<const char *>(b.p) + elems * eb) : nullptr;
    };
    while (a0 < v - 1) {
      const long per_a = static_cast<long>(v) * (v - a0) * v;
      long nA = std::max<long>(1, static_cast<long>(slab_budget / (per_a * veb)));
      nA = std::min<long>(nA, v - 1 - a0);
      const long a1 = a0 + nA;
      const long p0 = a0 * v - a0 * (a0 + 1) / 2;
      const long p1 = a1 * v - a1 * (a1 + 1) / 2;
      const long np = p1 - p0;
      if (Vs.bytes < veb * nA * per_a) Vs.reset(&al, veb * nA * per_a);
      if (Wh.bytes < eb * np * Kp2) {
        Wh.reset(&al, eb * np * Kp2);
        if (split) Wl.reset(&al, eb * np * Kp2);
      }
      TcDesc g1;
      g1.M = nA * v; g1.N = (v - a0) * v; g1.Kp = Kp1;
      g1.A = off(A1h, 2 * a0 * v * Kp1); g1.Alo = off(A1l, 2 * a0 * v * Kp1);
      g1.B = off(B1h, a0 * v * Kp1); g1.Blo = off(B1l, a0 * v * Kp1);
      g1.tier = tr; g1.out = TC_OUT_F32;
      g1.C = Vs.p; g1.ldc = (v - a0) * v;
      g1.amax_a = amx_L; g1.amax_b = amx_L;
      g1.amax_out = amx_W; g1.amax_mul = 2.0f;
      {
        Engine::Region r = eng.region("ladder gemm1");
        gemm_tc(g1, st, err_d.as<int>());
      }
      {
        Engine::Region r = eng.region("ladder antisym");
        ladder_antisym(Vs.p, true, v, static_cast<int>(a0), static_cast<int>(nA), p0, p1,
                       ab_a.as<int>(), ab_b.as<int>(), ab_a.as<int>(), ab_b.as<int>(), tr, Wh.p,
                       Wl.p, Kp2, nullptr, st, amx_W);
      }
      TcDesc g2;
      g2.M = n_ij; g2.N = np; g2.Kp = Kp2;
      g2.A = A2h.p; g2.Alo = A2l.p; g2.B = Wh.p; g2.Blo = Wl.p;
      g2.tier = tr; g2.out = TC_OUT_F64;
      g2.C = Rp.c() + p0; g2.ldc = n_ab;
      g2.amax_a = amx_t; g2.amax_b = amx_W;
      g2.bn = tc_pick_bn(np);
      g2.split_k = tc_pick_split(((2 * n_ij + 127) / 128) * ((np + g2.bn - 1) / g2.bn), Kp2 / kal,
                                 num_sms);
      if (g2.split_k > 1) {
        // partial sums accumulate atomically into this block's zeroed columns
        scale_2d(static_cast<cplx *>(g2.C), nullptr, nullptr, n_ab, n_ij, np, C0(), st);
        g2.out = TC_OUT_F64_ATOMIC;
      }
      {
        Engine::Region r = eng.region("ladder gemm2");
        gemm_tc(g2, st, err_d.as<int>());
      }
      a0 = a1;
    }
  }
  unpack_pairs_add(Rp.c(), o, v, ij_i.as<int>(), ij_j.as<int>(), ab_a.as<int>(), ab_b.as<int>(), R2,
                   st);
  CUDA_CHECK(cudaEventRecord(tm->e1, st));
  ladder_timing.push_back(tm);
  stat[2] = 8.0 * (static_cast<double>(X) * v * v * v * (v - 1) / 2.0 +
                   static_cast<double>(n_cd) * n_cd * n_ij);
}

void Ctx::settle_ladder_timing() {
  for (const auto &t : ladder_timing) {
    CUDA_CHECK(cudaEventSynchronize(t->e1));
    float ms = 0;
    CUDA_CHECK(cudaEventElapsedTime(&ms, t->e0, t->e1));
    stat[0] += ms;
    stat[1] += 1;
  }
  ladder_timing.clear();
}

// ===========================================================================
// CCSD residual (Eqs. 13-14, spin-orbital intermediate form)
// ===========================================================================
void Ctx::residual(const cplx *t1p, const cplx *t2p, cplx *R1, cplx *R2) {
  const int tr = res_tier();
  // the singles intermediates (matrix-vector shapes, memory bound): FP64 in
  // the FP64 tier, FP32 products summed in FP64 on the CUDA cores otherwise
  const int sx = tr == TIER_FP64 ? TIER_FP64 : TIER_SIMT32;
  const long oo = static_cast<long>(o) * o, vv = static_cast<long>(v) * v, n2 = oo * vv;
  Buf tau(&al, sizeof(cplx) * n2), taut(&al, sizeof(cplx) * n2);
  // FP16 tiers: the maximum of each doubles-sized operand, shared by all of
  // its uses ([0] t2, [1] tau, [2] tau~), found by the kernel that forms tau
  const bool scaled = tier_scaled(tr);
  Buf amx(&al, 3 * sizeof(float));
  float *amx_t2 = nullptr, *amx_tau = nullptr, *amx_taut = nullptr;
  if (scaled) {
    amx_t2 = amx.as<float>();
    amx_tau = amx_t2 + 1;
    amx_taut = amx_t2 + 2;
  }
  {
    Engine::Region r = eng.region("make_tau x2");
    make_tau_pair(t1p, t2p, tau.c(), taut.c(), o, v, st, tr != TIER_FP64, amx_t2);
  }
  auto t2 = [&](const char *ix) { return with_amax(T(t2p, ix, {o, o, v, v}), amx_t2); };
  // packed planes of t2 kept within this call are dropped on every way out
  struct ForgetPacks {
    Engine &e;
    const void *p;
    ~ForgetPacks() { e.forget_packs(p); }
  } forget_t2{eng, t2p};
  auto tauT = [&](const char *ix) { return with_amax(T(tau.c(), ix, {o, o, v, v}), amx_tau); };
  auto tautT = [&](const char *ix) { return with_amax(T(taut.c(), ix, {o, o, v, v}), amx_taut); };
  Buf Fae(&al, sizeof(cplx) * vv), Fmi(&al, sizeof(cplx) * oo), Fme(&al, sizeof(cplx) * o * v);
  Buf cP(&al, sizeof(cplx) * X), Y(&al, sizeof(cplx) * X * v * o), Zm(&al, sizeof(cplx) * X * oo);
  Buf Q(&al, sizeof(cplx) * X * o * v);
  const std::vector<long> d_oo = {o, o}, d_ov = {o, v}, d_vv = {v, v};
  auto t1 = [&](const char *ix) { return T(t1p, ix, {o, v}); };
  auto g_oovv = [&](const char *ix) { return stable(T(oovv.c(), ix, {o, o, v, v})); };
  auto g_ooov = [&](const char *ix) { return stable(T(ooov.c(), ix, {o, o, o, v})); };
  auto g_ovvo = [&](const char *ix) { return stable(T(ovvo.c(), ix, {o, v, v, o})); };
  auto Lov_ = [&](const char *ix) { return stable(T(Lov.c(), ix, {X, o, v})); };
  auto Lvo_ = [&](const char *ix) { return stable(T(Lvo.c(), ix, {X, v, o})); };
  auto Lvv_ = [&](const char *ix) { return stable(T(Lvv.c(), ix, {X, v, v})); };

  // F_me = sum_nf t_n^f <mn||ef>
  eng.contract(C1(), t1("nf"), g_oovv("mnef"), C0(), T(Fme.c(), "me", {o, v}), sx);
  // F_ae = sum_mf t_m^f <ma||fe> - 1/2 tau~_mn^af <mn||ef>; the first term
  // through L: sum_P c_P L^P_ae - sum_Pm L^P_me Y^P_am, Y^P_am = sum_f L^P_af t_m^f
  eng.contract(C1(), t1("mf"), Lov_("Pmf"), C0(), T(cP.c(), "P", {X}), sx);
  eng.contract(C1(), Lvv_("Paf"), t1("mf"), C0(), T(Y.c(), "Pam", {X, v, o}), tr);
  eng.contract(C1(), T(cP.c(), "P", {X}), Lvv_("Pae"), C0(), T(Fae.c(), "ae", {v, v}), sx);
  eng.contract(Cr(-1), Lov_("Pme"), T(Y.c(), "Pam", {X, v, o}), C1(), T(Fae.c(), "ae", {v, v}), tr);
  eng.contract(Cr(-0.5), tautT("mnaf"), g_oovv("mnef"), C1(),
               T(Fae.c(), "ae", {v, v}), tr);
  // F_mi = sum_ne t_n^e <mn||ie> + 1/2 tau~_in^ef <mn||ef>
  eng.contract(C1(), g_ooov("mnie"), t1("ne"), C0(), T(Fmi.c(), "mi", {o, o}), sx);
  eng.contract(Cr(0.5), g_oovv("mnef"), tautT("inef"), C1(),
               T(Fmi.c(), "mi", {o, o}), tr);
  taut.release();

  // ---------------- singles (Eq. 13) ----------------
  eng.contract(C1(), t1("ie"), T(Fae.c(), "ae", {v, v}), C0(), T(R1, "ia", {o, v}), sx);
  eng.contract(Cr(-1), t1("ma"), T(Fmi.c(), "mi", {o, o}), C1(), T(R1, "ia", {o, v}), sx);
  eng.contract(C1(), t2("imae"), T(Fme.c(), "me", {o, v}), C1(), T(R1, "ia", {o, v}), sx);
  eng.contract(C1(), t1("nf"), g_ovvo("nafi"), C1(), T(R1, "ia", {o, v}), sx);
  // -1/2 t_im^ef <ma||ef> = -sum_Pf L^P_af Q^P_if, Q^P_if = sum_me t_im^ef L^P_me
  // t2 with rows (i, f) and K (m, e): the same packed planes serve the ring
  // product below (rows (i, a), K (m, e)), so they are kept until then
  eng.contract(C1(), stable(t2("imef")), Lov_("Pme"), C0(), T(Q.c(), "Pif", {X, o, v}), tr);
  eng.contract(Cr(-1), Lvv_("Paf"), T(Q.c(), "Pif", {X, o, v}), C1(), T(R1, "ia", {o, v}), tr);
  // -1/2 t_mn^ae <nm||ei> = +1/2 t_mn^ae <nm||ie>
  eng.contract(Cr(0.5), t2("mnae"), g_ooov("nmie"), C1(), T(R1, "ia", {o, v}), tr);
  Q.release();

  // ---------------- doubles (Eq. 14) ----------------
  Buf Xb(&al, sizeof(cplx) * n2);
  auto Xt = [&](const char *ix) { return T(Xb.c(), ix, {o, o, v, v}); };
  auto R2t = [&](const char *ix) { return T(R2, ix, {o, o, v, v}); };
  // driver <ab||ij> = conj(<ij||ab>)
  eng.permute_into(C1(), conj(g_oovv("ijab")), C0(), R2t("ijab"));
  // Terms that need an antisymmetriser are summed into one scratch X, and a
  // single P(ij)P(ab) pass adds X to R2 at the end. A P(ab) term f that is
  // itself antisymmetric in (i, j) equals 1/2 P(ij)P(ab) f, and a P(ij) term
  // antisymmetric in (a, b) equals 1/2 P(ij)P(ab) of itself, so every
  // one-pair term enters X with a factor 1/2.
  // Hole-ladder intermediate W'_mnij = <mn||ij> + P(ij) t_j^e <mn||ie>,
  // antisymmetric in (m, n). The hole ladder 1/2 tau_mn^ab W'_mnij splits
  // into its t2 part (taken below with the Z term) and its t1 t1 part,
  // sum_mn t_m^a t_n^b W'_mnij, which is antisymmetric in (a, b): it joins
  // the P(ab) terms as 1/2 sum_mn t_m^a t_n^b W'_mnij.
  const std::initializer_list<long> d4 = {o, o, o, o};
  Buf Wp(&al, sizeof(cplx) * oo * oo);
  {
    Buf tmp(&al, sizeof(cplx) * oo * oo);
    d2d(Wp.p, oooo.p, sizeof(cplx) * oo * oo, st);
    eng.contract(C1(), g_ooov("mnie"), t1("je"), C0(), T(tmp.c(), "mnij", d4), tr);
    eng.permute_into(C1(), T(tmp.c(), "mnij", d4), C1(), T(Wp.c(), "mnij", d4));
    eng.permute_into(Cr(-1), T(tmp.c(), "mnji", d4), C1(), T(Wp.c(), "mnij", d4));
  }
  // P(ij) [-t_im^ab (F_mj + 1/2 t_j^e F_me)], antisymmetric in (a, b): the
  // first writer of X (plain stores; measured a little faster than taking
  // the tensor-core product below first)
  {
    Buf Fmj(&al, sizeof(cplx) * oo);
    d2d(Fmj.p, Fmi.p, sizeof(cplx) * oo, st);
    eng.contract(Cr(0.5), t1("je"), T(Fme.c(), "me", {o, v}), C1(), T(Fmj.c(), "mj", {o, o}),
                 sx);
    eng.contract(Cr(-0.5), t2("imab"), T(Fmj.c(), "mj", {o, o}), C0(), Xt("ijab"), tr);
  }
  // P(ab) [t_ij^ae (F_be - 1/2 t_m^b F_me) + sum_m t_m^a Q_ijmb] with
  // Q_ijmb = -<mb||ij> + 1/2 sum_n W'_mnij t_n^b, <mb||ij> = conj(<ij||mb>);
  // both parts are antisymmetric in (i, j). The P(ij)P(ab) term
  // -t_m^a y_mbij with y_mbij = sum_e t_i^e <mb||ej> has the same form, so
  // one product over m takes both: X += sum_m t_m^a (1/2 Q_ijmb - y_mbij).
  {
    Buf Fbe(&al, sizeof(cplx) * vv);
    d2d(Fbe.p, Fae.p, sizeof(cplx) * vv, st);
    eng.contract(Cr(-0.5), t1("mb"), T(Fme.c(), "me", {o, v}), C1(), T(Fbe.c(), "be", {v, v}),
                 sx);
    eng.contract(Cr(0.5), t2("ijae"), T(Fbe.c(), "be", {v, v}), C1(), Xt("ijab"), tr);
    Buf Qm(&al, sizeof(cplx) * oo * o * v);
    auto Qt = [&](const char *ix) { return T(Qm.c(), ix, {o, o, o, v}); };
    eng.permute_into(Cr(-0.5), conj(g_ooov("ijmb")), C0(), Qt("ijmb"));
    eng.contract(Cr(0.25), T(Wp.c(), "mnij", d4), t1("nb"), C1(), Qt("ijmb"), tr);
    {
      Buf y2(&al, sizeof(cplx) * oo * o * v);
      eng.contract(C1(), t1("ie"), g_ovvo("mbej"), C0(), T(y2.c(), "mbij", {o, v, o, o}), tr);
      eng.permute_into(Cr(-1), T(y2.c(), "mbij", {o, v, o, o}), C1(), Qt("ijmb"));
    }
    eng.contract(C1(), t1("ma"), Qt("ijmb"), C1(), Xt("ijab"), tr);
  }
  // P(ij) t_i^e <ab||ej> = P(ij)P(ab) T_ijab with T_ijab = sum_P Y^P_ai L^P_bj,
  // since t_i^e <ab||ej> = sum_P (Y^P_ai L^P_bj - L^P_aj Y^P_bi) = T_ijab - T_ijba
  eng.contract(C1(), T(Y.c(), "Pai", {X, v, o}), Lvo_("Pbj"), C1(), Xt("ijab"), tr);
  // hole ladder, t2 part: sum_mn t_mn^ab (1/2 W'_mnij + 1/4 Z_mnij), with
  // Z_mnij = sum_ef <mn||ef> tau_ij^ef
  {
    Buf Zb(&al, sizeof(cplx) * oo * oo);
    eng.contract(C1(), g_oovv("mnef"), tauT("ijef"), C0(), T(Zb.c(), "mnij", d4), tr);
    axpby(oo * oo, Cr(0.5), Wp.c(), Cr(0.25), Zb.c(), st);
    // (i,j) as the GEMM rows so the output rows (a,b) are contiguous
    eng.contract(C1(), T(Zb.c(), "mnij", d4), t2("mnab"), C1(), R2t("ijab"), tr);
  }
  Wp.release();
  // particle ladder with T1-dressed vectors: L~^P_ac = L^P_ac - sum_m t_m^a L^P_mc
  {
    Buf Lt(&al, sizeof(cplx) * X * vv);
    d2d(Lt.p, Lvv.p, sizeof(cplx) * X * vv, st);
    eng.contract(Cr(-1), t1("ma"), Lov_("Pmc"), C1(), T(Lt.c(), "Pac", {X, v, v}), tr);
    Engine::Region r = eng.region("ladder total");
    ladder(Lt.c(), tau.c(), R2, tr, amx_tau);
  }
  // W_mbej, stored as W[j][b][m][e]: its producers then write rows of
  // contiguous (m, e) and the ring contraction below reads contiguous K
  Buf W(&al, sizeof(cplx) * n2);
  auto Wt = [&](const char *ix) { return T(W.c(), ix, {o, v, o, v}); };  // "jbme" order
  if (ovvo_jbme.p)
    d2d(W.p, ovvo_jbme.p, sizeof(cplx) * n2, st);
  else
    eng.permute_into(C1(), g_ovvo("mbej"), C0(), Wt("jbme"));
  //   + t_j^f <mb||ef> = sum_P L^P_me Y^P_bj - sum_P Z^P_mj L^P_be
  eng.contract(C1(), T(Y.c(), "Pbj", {X, v, o}), Lov_("Pme"), C1(), Wt("jbme"), tr);
  eng.contract(C1(), Lov_("Pmf"), t1("jf"), C0(), T(Zm.c(), "Pmj", {X, o, o}), tr);
  eng.contract(Cr(-1), T(Zm.c(), "Pmj", {X, o, o}), Lvv_("Pbe"), C1(), Wt("jbme"), tr);
  //   - t_n^b <mn||ej> - t_j^f t_n^b <mn||ef> = t_n^b (<mn||je> - u_mnje)
  //   with u_mnje = sum_f <mn||ef> t_j^f: one product over n for both
  {
    const std::initializer_list<long> d3v = {o, o, o, v};
    Buf u(&al, sizeof(cplx) * oo * o * v);
    eng.contract(C1(), g_oovv("mnef"), t1("jf"), C0(), T(u.c(), "mnje", d3v), tr);
    axpby(oo * o * v, C1(), ooov.c(), Cr(-1), u.c(), st);
    eng.contract(C1(), T(u.c(), "mnje", d3v), t1("nb"), C1(), Wt("jbme"), tr);
  }
  //   - 1/2 t_jn^fb <mn||ef>
  eng.contract(Cr(-0.5), t2("jnfb"), g_oovv("mnef"), C1(), Wt("jbme"), tr);
  // P(ij)P(ab) [t_im^ae W_mbej - t_i^e t_m^a <mb||ej>], the second part
  // taken with the Q product above
  eng.contract(C1(), stable(t2("imae")), Wt("jbme"), C1(), Xt("ijab"), tr);
  eng.forget_packs(t2p);
  { Engine::Region r_ = eng.region("antisym_add"); antisym_add(R2, Xb.c(), o, v, 1.0, 3, st); }
}

// ===========================================================================
// CCSD iterations with Jacobi updates and DIIS
// ===========================================================================
size_t Ctx::planes_bytes_estimate(int tr) const {
  if (tr == TIER_FP64) return 0;
  // the largest doubles-sized contraction (M K = o^2 v^2, N <= M) packs its
  // A side into 2M x 2K and its B side into N x 2K elements of the tier's
  // type, twice for the hi/lo tiers
  const double mk = static_cast<double>(o) * o * v * v;
  return static_cast<size_t>(6.0 * mk * tc_elem_bytes(tr) * (tier_split(tr) ? 2 : 1));
}

size_t Ctx::residual_bytes_estimate() const {
  const double nb2 = static_cast<double>(sizeof(cplx)) * o * o * v * v;
  const double lvv = static_cast<double>(sizeof(cplx)) * X * v * v;
  return static_cast<size_t>(4 * nb2 + lvv) + planes_bytes_estimate(res_tier()) + slab_budget;
}

int Ctx::ccsd(double tol, int max_iter, double *e_out, int *n_iter) {
  if (!(tol > 0) || max_iter < 1) fail(CC_ERR_ARG, "tol must be > 0 and max_iter >= 1");
  ensure_ready();
  eng.clear_pack_cache();
  const double t0 = now_ms();
  const long n1 = static_cast<long>(o) * v, n2 = static_cast<long>(o) * o * v * v;
  const long na = n_amp();
  B(t1, n1);
  B(t2, n2);
  ensure_pairs();
  if (!amps) {
    mp2_amplitudes(oovv.c(), eps_d.as<double>(), o, v, t1.c(), t2.c(), st);
    amps = true;
  }
  Buf R1(&al, sizeof(cplx) * n1), R2(&al, sizeof(cplx) * n2);
  Buf vcur(&al, sizeof(cplx) * na), vnew(&al, sizeof(cplx) * na), step(&al, sizeof(cplx) * na);
  Buf invd(&al, sizeof(double) * na);
  // Device memory beyond the buffers above: the residual's transient buffers
  // must stay allocatable; what is left holds, in this order of preference,
  // the DIIS history (m_max pairs of packed vectors), the cache of packed
  // stable operands, and the <mb||ej> copy in the ring term's layout. On a
  // device with room for everything (all but the largest systems) all three
  // are kept; otherwise the copy is skipped, operands are packed on each use
  // and the DIIS history grows only as far as memory allows.
  const int m_max = 8, diis_start = 2;
  const size_t pair_bytes = 2 * sizeof(cplx) * na;
  size_t res_need = residual_bytes_estimate();
  eng.cache_reserve = res_need + m_max * pair_bytes;
  if (device_avail(&al) >= sizeof(cplx) * n2 + res_need + m_max * pair_bytes) {
    ovvo_jbme.reset(&al, sizeof(cplx) * n2);
    eng.permute_into(C1(), T(ovvo.c(), "mbej", {o, v, v, o}), C0(),
                     T(ovvo_jbme.c(), "jbme", {o, v, o, v}));
  }
  cc_tier = -1;
  cc_done_tier = -1;
  struct Release {
    Buf &b;
    Engine &e;
    int &t;
    ~Release() {
      b.release();
      e.cache_reserve = 0;
      t = -1;
    }
  } release_jbme{ovvo_jbme, eng, cc_tier};
  amp_denoms(eps_d.as<double>(), o, v, ij_i.as<int>(), ij_j.as<int>(), ab_a.as<int>(),
             ab_b.as<int>(), invd.as<double>(), st);
  const long esl = energy_scratch_len(o, v);
  Buf escr(&al, sizeof(cplx) * (esl + 1));
  const bool e32 = tier != TIER_FP64;
  auto energy_of = [&](const Buf &vec) {
    energy_packed(oovv.c(), vec.c(), o, v, ij_i.as<int>(), ij_j.as<int>(), ab_a.as<int>(),
                  ab_b.as<int>(), e32, escr.c(), esl, escr.c() + esl, st);
    cplx h;
    d2h(&h, escr.c() + esl, sizeof(cplx), st);
    return h;
  };
  std::vector<Buf> hv(m_max), he(m_max);
  Buf Bm(&al, sizeof(cplx) * 16 * 16), coef(&al, sizeof(cplx) * 16), dstat(&al, sizeof(int) * 4);
  int n_hist = 0, slot = 0, diis_cap = 0;
  size_t loop_peak = 0;  // device bytes held at most during the iterations
  // The one-product tiers (TF32, FP16) leave a floor under ||dt|| that
  // rises with the size of the amplitudes. When the best step norm has not
  // halved for three iterations, the remaining iterations run in the
  // tier's split form (TF32x3, FP16x3) and the DIIS history starts again
  // from errors of that residual.
  const int acc_tier = tier_accurate(tier);
  double best_step = HUGE_VAL;
  int since_best = 0, escalated_at = 0;
  std::vector<int> order;  // slots in age order
  pack_amps(t1.c(), t2.c(), o, v, ij_i.as<int>(), ij_j.as<int>(), ab_a.as<int>(), ab_b.as<int>(), vcur.c(), st);
  cplx e_old = energy_of(vcur);
  bool converged = false;
  int it = 0;
  for (it = 1; it <= max_iter; ++it) {
    {
      // the bytes this residual allocates beyond what it started with
      const size_t base = al.in_use;
      al.window = base;
      Engine::Region r = eng.region("residual total");
      residual(t1.c(), t2.c(), R1.c(), R2.c());
      maybe_inject(1, it, R2.c() + (o > 1 && v > 1 ? static_cast<long>(v) * v + 1 : 0));  // (0,1,0,1)
      res_need = al.window - base;
      loop_peak = std::max(loop_peak, al.window);
    }
    Engine::Region r_upd = eng.region("update+diis");
    jacobi_packed(R1.c(), R2.c(), invd.as<double>(), o, v, ij_i.as<int>(), ij_j.as<int>(),
                  ab_a.as<int>(), ab_b.as<int>(), vnew.c(), st);
    d2d(step.p, vnew.p, sizeof(cplx) * na, st);
    axpby(na, Cr(-1), vcur.c(), C1(), step.c(), st);
    const cplx nrm2 = dot(step.c(), step.c(), na, true, st, red.c());
    const double dnorm = std::sqrt(std::max(nrm2.x, 0.0));
    const cplx e_new = energy_of(vnew);
    check_err_flag();
    if (!std::isfinite(dnorm) || !std::isfinite(e_new.x) || !std::isfinite(e_new.y))
      fail(CC_ERR_NUMERIC, "CCSD iteration produced NaN/Inf");
    const double de = std::hypot(e_new.x - e_old.x, e_new.y - e_old.y);
    if (dnorm < tol && de < tol) {
      unpack_amps(vnew.c(), o, v, t1.c(), t2.c(), st);
      e_old = e_new;
      converged = true;
      break;
    }
    if (dnorm < 0.5 * best_step) {
      best_step = dnorm;
      since_best = 0;
    } else if (++since_best >= 3 && !escalated_at && acc_tier != tier) {
      escalated_at = it;
      cc_tier = acc_tier;
      eng.clear_pack_cache();  // packed in the one-product tier
      for (int k = 0; k < m_max; ++k) {
        hv[k].release();
        he[k].release();
      }
      n_hist = 0;
      diis_cap = 0;
      order.clear();
      best_step = HUGE_VAL;
      since_best = 0;
    }
    // a new history slot only while the next residual keeps room (the
    // step just taken in the one-product tier does not enter a history
    // restarted for the split tier)
    const bool use_diis = it >= diis_start && escalated_at != it;
    if (use_diis && n_hist < m_max && n_hist == diis_cap &&
        device_avail(&al) >= pair_bytes + res_need)
      ++diis_cap;
    if (use_diis && diis_cap > 0) {
      // push (vnew, step) into the ring of diis_cap slots
      if (n_hist < diis_cap) {
        slot = n_hist++;
        hv[slot].reset(&al, sizeof(cplx) * na);
        he[slot].reset(&al, sizeof(cplx) * na);
        order.push_back(slot);
      } else {
        slot = order.front();
        order.erase(order.begin());
        order.push_back(slot);
      }
      d2d(hv[slot].p, vnew.p, sizeof(cplx) * na, st);
      d2d(he[slot].p, step.p, sizeof(cplx) * na, st);
      // B[i][slot] = <e_i|e_slot>, B[slot][i] = conj
      {
        std::vector<const cplx *> xs(n_hist);
        for (int k = 0; k < n_hist; ++k) xs[k] = he[k].c();
        dot_multi(xs.data(), n_hist, he[slot].c(), na, tier != TIER_FP64, Bm.c() + slot, 16,
                  red.c(), 4096, st);
      }
      // mirror the new column into the new row (Hermitian)
      {
        std::vector<cplx> Bh(16 * 16);
        d2h(Bh.data(), Bm.p, sizeof(cplx) * 256, st);
        for (int k = 0; k < n_hist; ++k) Bh[slot * 16 + k] = cconj(Bh[k * 16 + slot]);
        // order the system by age so the solve is independent of slot layout
        std::vector<cplx> Bo(16 * 16);
        for (int a = 0; a < n_hist; ++a)
          for (int b = 0; b < n_hist; ++b) Bo[a * 16 + b] = Bh[order[a] * 16 + order[b]];
        h2d(Bm.p, Bh.data(), sizeof(cplx) * 256, st);
        if (n_hist >= 2) {
          Buf Bord(&al, sizeof(cplx) * 256);
          h2d(Bord.p, Bo.data(), sizeof(cplx) * 256, st);
          diis_solve(Bord.c(), n_hist, 16, coef.c(), dstat.as<int>(), st);
          int ds = 0;
          d2h(&ds, dstat.p, sizeof(int), st);
          if (ds == 0) {
            std::vector<cplx *> vp(n_hist);
            for (int a = 0; a < n_hist; ++a) vp[a] = hv[order[a]].c();
            diis_combine(vp.data(), coef.c(), n_hist, na, vnew.c(), st);
          }
        }
      }
    }
    unpack_amps(vnew.c(), o, v, t1.c(), t2.c(), st);
    d2d(vcur.p, vnew.p, sizeof(cplx) * na, st);
    e_old = energy_of(vnew);
  }
  if (it > max_iter) it = max_iter;
  e_corr = e_old;
  if (e_out) {
    e_out[0] = e_corr.x;
    e_out[1] = e_corr.y;
  }
  if (n_iter) *n_iter = it;
  eng.trace_flush();
  settle_ladder_timing();
  stat[4] += now_ms() - t0;
  stat[7] = it;
  stat[13] = static_cast<double>(loop_peak);
  stat[15] = escalated_at;
  diis_depth = n_hist;
  cc_done_tier = res_tier();
  ccsd_done = true;
  hbar_done = false;
  return converged ? CC_OK : CC_ERR_NOT_CONVERGED;
}

// ===========================================================================
// H-bar elements with at most two virtual indices (built once)
// ===========================================================================
void Ctx::build_hbar() {
  Engine::Region rg = eng.region("hbar total");
  eng.clear_pack_cache();
  // packed operands are cached while tau, Q, the <mb||ej> - Q copy, the
  // (me|bf) block and the operand planes stay allocatable
  eng.cache_reserve = static_cast<size_t>(3.0 * sizeof(cplx) * o * o * v * v) +
                      planes_bytes_estimate(hbar_tier()) + slab_budget;
  struct ResetReserve {
    Engine &e;
    ~ResetReserve() { e.cache_reserve = 0; }
  } reset_reserve{eng};
  ++sig_gen;
  const int tr = hbar_tier();
  const int sx = tr == TIER_FP64 ? TIER_FP64 : TIER_SIMT32;
  const long oo = static_cast<long>(o) * o, vv = static_cast<long>(v) * v, ov = static_cast<long>(o) * v;
  const long n2 = oo * vv;
  // the amplitudes, tau and the integrals stay fixed during the build: their
  // packed tensor-core planes are made once (the pack cache is cleared on
  // entry and on exit); t2 and tau carry the maxima found while forming tau
  const bool scaled = tier_scaled(tr);
  Buf hmx(&al, 3 * sizeof(float)), gmx(&al, sizeof(float));
  const float *amx_t2 = scaled ? hmx.as<float>() : nullptr;
  const float *amx_tau = scaled ? hmx.as<float>() + 1 : nullptr;
  auto a1 = [&](const char *ix) { return T(t1.c(), ix, {o, v}); };
  auto t2t = [&](const char *ix) { return stable(with_amax(T(t2.c(), ix, {o, o, v, v}), amx_t2)); };
  auto g_oovv = [&](const char *ix) { return stable(T(oovv.c(), ix, {o, o, v, v})); };
  auto g_ooov = [&](const char *ix) { return stable(T(ooov.c(), ix, {o, o, o, v})); };
  auto Lov_ = [&](const char *ix) { return stable(T(Lov.c(), ix, {X, o, v})); };
  auto Lvv_ = [&](const char *ix) { return stable(T(Lvv.c(), ix, {X, v, v})); };
  const std::initializer_list<long> d4 = {o, o, o, o};
  Buf tau(&al, sizeof(cplx) * n2), Qh;
  make_tau(t1.c(), t2.c(), tau.c(), o, v, 1.0, st, tr != TIER_FP64, scaled ? hmx.as<float>() : nullptr);
  auto tauH = [&](const char *ix) { return stable(with_amax(T(tau.c(), ix, {o, o, v, v}), amx_tau)); };
  B(Hov, ov);
  B(Hoo, oo);
  B(Hvv, vv);
  B(Hoooo, oo * oo);
  B(Hooov, oo * ov);
  B(Hovvo, n2);
  B(Hovoo, oo * ov);
  // H_me
  eng.contract(C1(), a1("nf"), g_oovv("mnef"), C0(), T(Hov.c(), "me", {o, v}), sx);
  // H_mi = f_mi + t_n^e <mn||ie> + 1/2 tau_in^ef <mn||ef>
  eng.contract(C1(), g_ooov("mnie"), a1("ne"), C0(), T(Hoo.c(), "mi", {o, o}), sx);
  eng.contract(Cr(0.5), g_oovv("mnef"), tauH("inef"), C1(),
               T(Hoo.c(), "mi", {o, o}), tr);
  add_diag(Hoo.c(), eps_d.as<double>(), o, st);
  // H_ae = f_ae + t_m^f <am||ef> - 1/2 tau_mn^af <mn||ef>
  {
    Buf cP(&al, sizeof(cplx) * X), Y(&al, sizeof(cplx) * X * v * o);
    eng.contract(C1(), a1("mf"), Lov_("Pmf"), C0(), T(cP.c(), "P", {X}), sx);
    eng.contract(C1(), Lvv_("Paf"), a1("mf"), C0(), T(Y.c(), "Pam", {X, v, o}), tr);
    eng.contract(C1(), T(cP.c(), "P", {X}), Lvv_("Pae"), C0(), T(Hvv.c(), "ae", {v, v}), sx);
    eng.contract(Cr(-1), Lov_("Pme"), T(Y.c(), "Pam", {X, v, o}), C1(), T(Hvv.c(), "ae", {v, v}), tr);
    eng.contract(Cr(-0.5), tauH("mnaf"), g_oovv("mnef"), C1(),
                 T(Hvv.c(), "ae", {v, v}), tr);
    add_diag(Hvv.c(), eps_d.as<double>() + o, v, st);
    // H_mbej = <mb||ej> + t_j^f <mb||ef> - t_n^b <mn||ej> - (t_jn^fb + t_j^f t_n^b) <mn||ef>
    d2d(Hovvo.p, ovvo.p, sizeof(cplx) * n2, st);
    auto Ht = [&](const char *ix) { return T(Hovvo.c(), ix, {o, v, v, o}); };
    eng.contract(C1(), Lov_("Pme"), T(Y.c(), "Pbj", {X, v, o}), C1(), Ht("mbej"), tr);
    Buf Zm(&al, sizeof(cplx) * X * oo);
    eng.contract(C1(), Lov_("Pmf"), a1("jf"), C0(), T(Zm.c(), "Pmj", {X, o, o}), tr);
    eng.contract(Cr(-1), T(Zm.c(), "Pmj", {X, o, o}), Lvv_("Pbe"), C1(), Ht("mbej"), tr);
    eng.contract(C1(), g_ooov("mnje"), a1("nb"), C1(), Ht("mbej"), tr);
    // - (t_jn^fb + t_j^f t_n^b) <mn||ef> = - Q_mbej - t_n^b u_mnej with
    // Q_mbej = sum_nf t_jn^fb <mn||ef> (also used for H_mbij below) and
    // u_mnej = sum_f <mn||ef> t_j^f
    Qh.reset(&al, sizeof(cplx) * n2);
    eng.contract(C1(), g_oovv("mnef"), t2t("jnfb"), C0(), T(Qh.c(), "mbej", {o, v, v, o}), tr);
    axpby(n2, Cr(-1), Qh.c(), C1(), Hovvo.c(), st);
    Buf u(&al, sizeof(cplx) * oo * ov);
    eng.contract(C1(), g_oovv("mnef"), a1("jf"), C0(), T(u.c(), "mnej", {o, o, v, o}), tr);
    eng.contract(Cr(-1), a1("nb"), T(u.c(), "mnej", {o, o, v, o}), C1(), Ht("mbej"), tr);
  }
  // H_mnij = <mn||ij> + P(ij) t_j^e <mn||ie> + 1/2 tau_ij^ef <mn||ef>
  {
    Buf tmp(&al, sizeof(cplx) * oo * oo);
    d2d(Hoooo.p, oooo.p, sizeof(cplx) * oo * oo, st);
    eng.contract(C1(), g_ooov("mnie"), a1("je"), C0(), T(tmp.c(), "mnij", d4), tr);
    eng.permute_into(C1(), T(tmp.c(), "mnij", d4), C1(), T(Hoooo.c(), "mnij", d4));
    eng.permute_into(Cr(-1), T(tmp.c(), "mnji", d4), C1(), T(Hoooo.c(), "mnij", d4));
    eng.contract(Cr(0.5), g_oovv("mnef"), tauH("ijef"), C1(),
                 T(Hoooo.c(), "mnij", d4), tr);
  }
  // H_mnie = <mn||ie> + t_i^f <mn||fe>
  d2d(Hooov.p, ooov.p, sizeof(cplx) * oo * ov, st);
  eng.contract(C1(), g_oovv("mnfe"), a1("if"), C1(), T(Hooov.c(), "mnie", {o, o, o, v}), tr);
  // H_mbij = <mb||ij> - H_me t_ij^be - t_n^b H_mnij + 1/2 <mb||ef> tau_ij^ef
  //          + P(ij) [<mn||ie> t_jn^be + t_i^e (<mb||ej> - t_nj^bf <mn||ef>)]
  {
    auto Hb = [&](const char *ix) { return T(Hovoo.c(), ix, {o, v, o, o}); };
    eng.permute_into(C1(), conj(g_ooov("ijmb")), C0(), Hb("mbij"));
    eng.contract(Cr(-1), T(Hov.c(), "me", {o, v}), t2t("ijbe"), C1(), Hb("mbij"), tr);
    eng.contract(Cr(-1), a1("nb"), T(Hoooo.c(), "mnij", d4), C1(), Hb("mbij"), tr);
    // 1/2 <mb||ef> tau_ij^ef = sum_ef (me|bf) tau_ij^ef, (me|bf) formed from L
    // for a block of m at a time (three-virtual integrals never stored whole)
    const size_t per_m = sizeof(cplx) * static_cast<size_t>(v) * vv;
    const int mb = static_cast<int>(std::max<size_t>(1, std::min<size_t>(o, slab_budget / per_m)));
    Buf G(&al, per_m * mb);
    for (int m0 = 0; m0 < o; m0 += mb) {
      const int mc = std::min(mb, o - m0);
      // the GEMM writing the block records its maximum for the next one's scale
      eng.contract(C1(), Tv(Lov.c() + static_cast<long>(m0) * v, "Pme", {X, mc, v}, {ov, v, 1}),
                   Lvv_("Pbf"), C0(),
                   with_amax_out(T(G.c(), "mebf", {mc, v, v, v}), scaled ? gmx.as<float>() : nullptr),
                   tr);
      eng.contract(C1(), with_amax(T(G.c(), "mebf", {mc, v, v, v}), scaled ? gmx.as<float>() : nullptr),
                   tauH("ijef"), C1(),
                   T(Hovoo.c() + static_cast<long>(m0) * v * oo, "mbij", {mc, v, o, o}), tr);
    }
    G.release();
    Buf tW(&al, sizeof(cplx) * n2), y(&al, sizeof(cplx) * oo * ov);
    // <mb||ej> - t_nj^bf <mn||ef> = <mb||ej> - Q_mbej
    d2d(tW.p, ovvo.p, sizeof(cplx) * n2, st);
    axpby(n2, Cr(-1), Qh.c(), C1(), tW.c(), st);
    Qh.release();
    eng.contract(C1(), g_ooov("mnie"), t2t("jnbe"), C0(), T(y.c(), "mbij", {o, v, o, o}), tr);
    eng.contract(C1(), a1("ie"), T(tW.c(), "mbej", {o, v, v, o}), C1(), T(y.c(), "mbij", {o, v, o, o}),
                 tr);
    eng.permute_into(C1(), T(y.c(), "mbij", {o, v, o, o}), C1(), Hb("mbij"));
    eng.permute_into(Cr(-1), T(y.c(), "mbji", {o, v, o, o}), C1(), Hb("mbij"));
  }
  B(Hoo_off, oo);
  B(Hvv_off, vv);
  B(doo, o);
  B(dvv, v);
  split_diag(Hoo.c(), o, Hoo_off.c(), doo.c(), st);
  split_diag(Hvv.c(), v, Hvv_off.c(), dvv.c(), st);
  CUDA_CHECK(cudaStreamSynchronize(st));
  check_err_flag();
  // the sigma packs its operands in the EOM tier: the H-bar build's packed
  // planes are not used again
  eng.clear_pack_cache();
  hbar_done = true;
}

// ===========================================================================
// IP-EOM-CCSD (Eqs. 17-18): sigma and Davidson live in eom.cu
// ===========================================================================
void Ctx::sigma(int k, const cplx *r, cplx *s) {
  std::vector<Ctx *> one{this};
  batch_sigma(one, {k}, {r}, {s}, false);
  settle_sigma_timing();
}

void Ctx::left_sigma(int k, const cplx *l, cplx *s) {
  std::vector<Ctx *> one{this};
  batch_left_sigma(one, {k}, {l}, {s});
}

namespace {

// In-place inverse of a small complex matrix (Gauss-Jordan, partial
// pivoting); false when a pivot vanishes.
bool invert_small(std::vector<cplx> &a, int n) {
  std::vector<cplx> inv(static_cast<size_t>(n) * n, mk(0, 0));
  for (int i = 0; i < n; ++i) inv[i * n + i] = mk(1, 0);
  double scale = 0;
  for (const cplx &x : a) scale = std::max(scale, std::hypot(x.x, x.y));
  for (int col = 0; col < n; ++col) {
    int piv = col;
    double best = 0;
    for (int r = col; r < n; ++r) {
      const double m = std::hypot(a[r * n + col].x, a[r * n + col].y);
      if (m > best) {
        best = m;
        piv = r;
      }
    }
    if (!(best > 1e-12 * scale)) return false;
    if (piv != col)
      for (int j = 0; j < n; ++j) {
        std::swap(a[piv * n + j], a[col * n + j]);
        std::swap(inv[piv * n + j], inv[col * n + j]);
      }
    const cplx p = a[col * n + col];
    const double d = p.x * p.x + p.y * p.y;
    const cplx pinv = mk(p.x / d, -p.y / d);
    for (int j = 0; j < n; ++j) {
      a[col * n + j] = cmul(pinv, a[col * n + j]);
      inv[col * n + j] = cmul(pinv, inv[col * n + j]);
    }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const cplx f = a[r * n + col];
      for (int j = 0; j < n; ++j) {
        a[r * n + j] = csub(a[r * n + j], cmul(f, a[col * n + j]));
        inv[r * n + j] = csub(inv[r * n + j], cmul(f, inv[col * n + j]));
      }
    }
  }
  a = inv;
  return true;
}

}  // namespace

// Right vectors by the block Davidson of Eq. 18, left vectors (Eq. 20) by
// the same Davidson on the transposed sigma, then L <- (L^T R)^-1 L so that
// the pairs are biorthonormal over the nr roots (Eq. 19); this also
// separates degenerate roots and any difference in the order of ties.
int Ctx::ipeom_lr(int nr, double tol, int max_iter, double *omega, cplx *R_dev, cplx *L_dev,
                  int *n_iter) {
  if (!(tol > 0) || max_iter < 1) fail(CC_ERR_ARG, "tol must be > 0 and max_iter >= 1");
  std::vector<Ctx *> one{this};
  const long dim = dim_ip();
  int st_r = CC_OK, st_l = CC_OK, it_r = 0, it_l = 0;
  std::vector<double> wl(2 * static_cast<size_t>(nr));
  Buf Lraw(&al, sizeof(cplx) * nr * dim);
  const std::vector<cplx *> pr{R_dev}, pl{Lraw.c()};
  run_ipeom(one, nr, tol, max_iter, omega, nullptr, &it_r, &st_r, use_graphs, false, &pr);
  run_ipeom(one, nr, tol, max_iter, wl.data(), nullptr, &it_l, &st_l, false, true, &pl);
  if (n_iter) {
    n_iter[0] = it_r;
    n_iter[1] = it_l;
  }
  // S[k][l] = l_k . r_l (bilinear), A = S^-1, L = A Lraw
  Buf S(&al, sizeof(cplx) * nr * nr);
  eng.contract(C1(), T(Lraw.c(), "kd", {nr, dim}), T(R_dev, "ld", {nr, dim}), C0(),
               T(S.c(), "kl", {nr, nr}), TIER_FP64);
  std::vector<cplx> a(static_cast<size_t>(nr) * nr);
  d2h(a.data(), S.p, sizeof(cplx) * nr * nr, st);
  if (!invert_small(a, nr))
    fail(CC_ERR_NUMERIC, "left and right IP vectors cannot be made biorthonormal");
  h2d(S.p, a.data(), sizeof(cplx) * nr * nr, st);
  eng.contract(C1(), T(S.c(), "kj", {nr, nr}), T(Lraw.c(), "jd", {nr, dim}), C0(),
               T(L_dev, "kd", {nr, dim}), TIER_FP64);
  CUDA_CHECK(cudaStreamSynchronize(st));
  check_err_flag();
  return (st_r == CC_OK && st_l == CC_OK) ? CC_OK : CC_ERR_NOT_CONVERGED;
}

int Ctx::ipeom(int nr, double tol, int max_iter, double *omega, double *r1w, int *n_iter) {
  if (!(tol > 0) || max_iter < 1) fail(CC_ERR_ARG, "tol must be > 0 and max_iter >= 1");
  std::vector<Ctx *> one{this};
  int status = CC_OK;
  // keep the right vectors (training samples for the learned start)
  if (nr >= 1 && nr <= dim_ip() && last_R.bytes < sizeof(cplx) * nr * dim_ip())
    last_R.reset(&al, sizeof(cplx) * nr * dim_ip());
  last_nr = 0;
  std::vector<cplx *> vecs{last_R.c()};
  run_ipeom(one, nr, tol, max_iter, omega, r1w, n_iter, &status, use_graphs, false, &vecs);
  if (status == CC_OK) last_nr = nr;
  return status;
}

}  // namespace cdfns
