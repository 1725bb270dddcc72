// IP-EOM-CCSD eigenproblem (Eqs. 17-18) for one or several systems.
//
// Sigma is built for every system of a batch together: the small terms run
// directly, then the six dominant two-body terms of every system (uneven
// sizes allowed) go to ONE grouped persistent tensor-core launch, then a
// combine kernel per system. The whole batched sigma is captured once per
// (systems, vector counts) into a CUDA graph and replayed afterwards.
// The block Davidson of each system runs as a state machine, all systems in
// lockstep so that their sigma requests are served by one batched build.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <mutex>
#include <numeric>

#include "solver.h"

namespace cdfns {

void geev_dev(Allocator *al, cudaStream_t st, cplx *A, int m, cplx *w, cplx *vr);

namespace {

double now_ms() {
  return std::chrono::duration<double, std::milli>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

void d2h(void *dst, const void *src, size_t n, cudaStream_t st) {
  CUDA_CHECK(cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, st));
  CUDA_CHECK(cudaStreamSynchronize(st));
}
void h2d(void *dst, const void *src, size_t n, cudaStream_t st) {
  CUDA_CHECK(cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, st));
}
void d2d(void *dst, const void *src, size_t n, cudaStream_t st) {
  CUDA_CHECK(cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToDevice, st));
}

// ---------------------------------------------------------------------------
// graph cache
// ---------------------------------------------------------------------------
struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  unsigned long long launches = 0;
  std::vector<double> flops;  // algorithmic flops of each system's contractions
};
std::mutex g_graph_mu;
std::map<std::vector<long>, GraphEntry> g_graphs;
cudaStream_t g_cap_stream = nullptr;

cudaStream_t capture_stream() {
  if (!g_cap_stream) CUDA_CHECK(cudaStreamCreateWithFlags(&g_cap_stream, cudaStreamNonBlocking));
  return g_cap_stream;
}

// dst = src / |src| from the squared norm n2 (a device value, its real
// part), or zero when |src| < thr: the Davidson's normalisation decided on
// the device, so a block of new vectors needs no host round trip per vector.
__global__ void normalize_or_zero_kernel(double2 *__restrict__ dst, const double2 *__restrict__ src,
                                         long n, const double2 *__restrict__ n2, double thr) {
  const double nn = sqrt(fmax(n2->x, 0.0));
  const bool keep = !(nn < thr);
  const double s = keep ? 1.0 / nn : 0.0;
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    const double2 x = src[i];
    dst[i] = keep ? make_double2(x.x * s, x.y * s) : make_double2(0.0, 0.0);
  }
}

void normalize_or_zero(cplx *dst, const cplx *src, long n, const cplx *n2, double thr,
                       cudaStream_t st) {
  const unsigned blocks = static_cast<unsigned>(std::min<long>((n + 255) / 256, 4096));
  normalize_or_zero_kernel<<<blocks, 256, 0, st>>>(dst, src, n, n2, thr);
  LAUNCH_CHECK();
  count_launch();
}

}  // namespace

// Drop every graph that refers to ctx (called when a context goes away).
void drop_graphs(const void *ctx) {
  std::lock_guard<std::mutex> lk(g_graph_mu);
  for (auto it = g_graphs.begin(); it != g_graphs.end();) {
    bool hit = false;
    for (size_t i = 0; i + 2 < it->first.size(); i += 3)
      if (it->first[i] == reinterpret_cast<long>(ctx)) hit = true;
    if (hit) {
      cudaGraphExecDestroy(it->second.exec);
      it = g_graphs.erase(it);
    } else {
      ++it;
    }
  }
}

// ---------------------------------------------------------------------------
// batched sigma
// ---------------------------------------------------------------------------
namespace {

void ensure_ws(Ctx &c, long k) {
  auto &w = c.sws;
  if (w.kcap >= k) return;
  const long dim = c.dim_ip(), oo = static_cast<long>(c.o) * c.o, t = k * oo * c.v;
  const size_t z = sizeof(cplx);
  w.rin.reset(&c.al, z * k * dim);
  w.sout.reset(&c.al, z * k * dim);
  w.r1.reset(&c.al, z * k * c.o);
  w.s1.reset(&c.al, z * k * c.o);
  w.xe.reset(&c.al, z * k * c.v);
  for (Buf *b : {&w.r2, &w.s2, &w.tA, &w.tB, &w.tC, &w.X1, &w.X2}) b->reset(&c.al, z * t);
  w.kcap = k;
  ++c.sig_gen;
}

// Sigma for k[i] vectors of system i, read from sys[i]->sws.rin, written to
// sys[i]->sws.sout, all work on stream st.
void sigma_body(std::vector<Ctx *> &sys, const std::vector<int> &k, cudaStream_t st) {
  std::vector<TcDesc> descs;
  for (size_t q = 0; q < sys.size(); ++q) {
    Ctx &c = *sys[q];
    const int kk = k[q];
    if (kk == 0) continue;
    const int o = c.o, v = c.v, tr = c.eom();
    auto &w = c.sws;
    auto R1 = [&](const char *ix) { return T(w.r1.c(), ix, {kk, o}); };
    auto R2 = [&](const char *ix) { return T(w.r2.c(), ix, {kk, o, o, v}); };
    auto K4 = [&](const Buf &b, const char *ix) { return T(b.c(), ix, {kk, o, o, v}); };
    auto S1 = [&](const char *ix) { return T(w.s1.c(), ix, {kk, o}); };
    ip_unpack(w.rin.c(), kk, o, v, w.r1.c(), w.r2.c(), st);
    // 1h and the three-body intermediate: small, run directly
    c.eng.contract(Cr(-1), R1("Km"), T(c.Hoo_off.c(), "mi", {o, o}), C0(), S1("Ki"), TIER_FP64);
    c.eng.contract(C1(), R2("Kime"), T(c.Hov.c(), "me", {o, v}), C1(), S1("Ki"), TIER_FP64);
    c.eng.contract(Cr(-0.5), R2("Kmne"), stable(T(c.Hooov.c(), "mnie", {o, o, o, v})), C1(), S1("Ki"),
                   tr);
    c.eng.contract(Cr(0.5), R2("Kmnf"), stable(T(c.oovv.c(), "mnef", {o, o, v, v})), C0(),
                   T(w.xe.c(), "Ke", {kk, v}), tr);
    // 2h1p two-body terms, each into its own buffer, prepared for one launch
    TcDesc d;
    auto add = [&](bool p) {
      if (p) descs.push_back(d);
    };
    add(c.eng.prepare(Cr(-1), R1("Km"), stable(T(c.Hovoo.c(), "mbij", {o, v, o, o})), C0(),
                      K4(w.s2, "Kijb"), tr, 0, &d));
    add(c.eng.prepare(C1(), R2("Kije"), stable(T(c.Hvv_off.c(), "be", {v, v})), C0(),
                      K4(w.tA, "Kijb"), tr, 1, &d));
    add(c.eng.prepare(C1(), stable(T(c.Hoo_off.c(), "mi", {o, o})), R2("Kmjb"), C0(),
                      K4(w.X1, "Kijb"), tr, 2, &d));
    add(c.eng.prepare(Cr(0.5), R2("Kmnb"), stable(T(c.Hoooo.c(), "mnij", {o, o, o, o})), C0(),
                      K4(w.tB, "Kijb"), tr, 3, &d));
    add(c.eng.prepare(C1(), R2("Kime"), stable(T(c.Hovvo.c(), "mbej", {o, v, v, o})), C0(),
                      K4(w.X2, "Kijb"), tr, 4, &d));
    add(c.eng.prepare(Cr(-1), T(w.xe.c(), "Ke", {kk, v}), stable(T(c.t2.c(), "ijeb", {o, o, v, v})),
                      C0(), K4(w.tC, "Kijb"), tr, 5, &d));
  }
  if (!descs.empty()) gemm_tc_grouped(descs, st, sys[0]->err_d.as<int>());
  for (size_t q = 0; q < sys.size(); ++q) {
    Ctx &c = *sys[q];
    const int kk = k[q];
    if (kk == 0) continue;
    auto &w = c.sws;
    sigma_combine(w.s2.c(), w.tA.c(), w.tB.c(), w.tC.c(), w.X1.c(), w.X2.c(), kk, c.o, c.v, st);
    ip_diag_apply(w.r1.c(), w.r2.c(), c.doo.c(), c.dvv.c(), kk, c.o, c.v, w.s1.c(), w.s2.c(), st);
    ip_pack(w.s1.c(), w.s2.c(), kk, c.o, c.v, w.sout.c(), st);
  }
}

}  // namespace

// Sigma vectors for several systems at once: s[q] (k[q] x dim) = H-bar r[q].
void batch_sigma(std::vector<Ctx *> &sys, const std::vector<int> &k,
                 const std::vector<const cplx *> &r, const std::vector<cplx *> &s, bool use_graph) {
  const cudaStream_t user = sys[0]->st;
  const cudaStream_t cs = capture_stream();
  cudaEvent_t ev;
  CUDA_CHECK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  CUDA_CHECK(cudaEventRecord(ev, user));
  CUDA_CHECK(cudaStreamWaitEvent(cs, ev, 0));
  std::vector<cudaStream_t> saved(sys.size());
  std::vector<long> key;
  for (size_t q = 0; q < sys.size(); ++q) {
    Ctx &c = *sys[q];
    if (!c.hbar_done) c.build_hbar();
    ensure_ws(c, std::max(1, k[q]));
    saved[q] = c.eng.st;
    c.eng.st = cs;
    if (k[q]) d2d(c.sws.rin.p, r[q], sizeof(cplx) * k[q] * c.dim_ip(), cs);
  }
  auto make_key = [&]() {
    std::vector<long> kk;
    for (size_t q = 0; q < sys.size(); ++q) {
      kk.push_back(reinterpret_cast<long>(sys[q]));
      kk.push_back(k[q]);
      kk.push_back(sys[q]->sig_gen * 1000003L + sys[q]->eng.gen);
    }
    return kk;
  };
  key = make_key();
  // device time of the sigma build (the statistics of every system in the
  // batch are charged with it) and its algorithmic flops per system
  auto tm = std::make_shared<Ctx::EventPair>();
  CUDA_CHECK(cudaEventCreate(&tm->e0));
  CUDA_CHECK(cudaEventCreate(&tm->e1));
  CUDA_CHECK(cudaEventRecord(tm->e0, cs));
  std::vector<double> fl(sys.size(), 0.0);
  try {
    GraphEntry *ge = nullptr;
    if (use_graph) {
      std::lock_guard<std::mutex> lk(g_graph_mu);
      auto it = g_graphs.find(key);
      if (it != g_graphs.end()) ge = &it->second;
    }
    if (ge) {
      CUDA_CHECK(cudaGraphLaunch(ge->exec, cs));
      count_launch(ge->launches);
      fl = ge->flops;
    } else {
      // run once directly (allocates and packs whatever is new), then capture
      const unsigned long long l0 = t_launches;
      for (size_t q = 0; q < sys.size(); ++q) fl[q] = -sys[q]->eng.flops;
      sigma_body(sys, k, cs);
      for (size_t q = 0; q < sys.size(); ++q) fl[q] += sys[q]->eng.flops;
      const unsigned long long nl = t_launches - l0;
      if (use_graph) {
        // The direct pass may have (re)allocated buffers: key the graph on
        // the generations after it. A capture that fails leaves no graph and
        // the direct pass's results stand.
        key = make_key();
        cudaGraph_t graph = nullptr;
        bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
          try {
            sigma_body(sys, k, cs);
          } catch (...) {
            ok = false;
          }
          if (cudaStreamEndCapture(cs, &graph) != cudaSuccess) ok = false;
        }
        GraphEntry e;
        if (ok && graph && cudaGraphInstantiate(&e.exec, graph, 0) == cudaSuccess &&
            make_key() == key) {
          e.launches = nl;
          e.flops = fl;
          std::lock_guard<std::mutex> lk(g_graph_mu);
          g_graphs[key] = e;
        } else if (e.exec) {
          cudaGraphExecDestroy(e.exec);
        }
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        // the captured pass did not run
        g_launches -= t_launches - (l0 + nl);
        t_launches = l0 + nl;
      }
    }
  } catch (...) {
    for (size_t q = 0; q < sys.size(); ++q) sys[q]->eng.st = saved[q];
    cudaEventDestroy(ev);
    throw;
  }
  CUDA_CHECK(cudaEventRecord(tm->e1, cs));
  for (size_t q = 0; q < sys.size(); ++q) {
    sys[q]->sig_timing.push_back(tm);
    sys[q]->stat[18] += fl[q];
    sys[q]->stat[19] += k[q];
  }
  for (size_t q = 0; q < sys.size(); ++q) {
    Ctx &c = *sys[q];
    c.eng.st = saved[q];
    if (k[q]) d2d(s[q], c.sws.sout.p, sizeof(cplx) * k[q] * c.dim_ip(), cs);
  }
  CUDA_CHECK(cudaEventRecord(ev, cs));
  CUDA_CHECK(cudaStreamWaitEvent(user, ev, 0));
  CUDA_CHECK(cudaEventDestroy(ev));
}

// ---------------------------------------------------------------------------
// left sigma (Eqs. 19-20)
// ---------------------------------------------------------------------------
namespace {

// s = l^T H-bar_IP for kk packed left vectors, in the same layout as sigma's
// vectors. Eq. 19 pairs left and right vectors bilinearly over the unique
// elements, so this is the transpose of sigma_body's map: each of its terms
// is read with input and output exchanged, into G[K][p][q][b] (which is not
// antisymmetric in p, q); the packed result is G - G(p<->q), plus the
// one-body diagonal, which the transposition leaves unchanged.
void left_sigma_body(Ctx &c, int kk, const cplx *lin, cplx *sout) {
  const int o = c.o, v = c.v, tr = c.eom();
  const cudaStream_t st = c.st;
  auto &w = c.sws;
  auto L1 = [&](const char *ix) { return T(w.r1.c(), ix, {kk, o}); };
  auto L2 = [&](const char *ix) { return T(w.r2.c(), ix, {kk, o, o, v}); };
  auto G = [&](const char *ix) { return T(w.tA.c(), ix, {kk, o, o, v}); };
  auto S1 = [&](const char *ix) { return T(w.s1.c(), ix, {kk, o}); };
  auto S2 = [&](const char *ix) { return T(w.s2.c(), ix, {kk, o, o, v}); };
  ip_unpack(lin, kk, o, v, w.r1.c(), w.r2.c(), st);
  // 1h: -sum_i H_mi l_i - 1/2 sum_bij H_mbij l_ij^b
  c.eng.contract(Cr(-1), L1("Ki"), T(c.Hoo_off.c(), "mi", {o, o}), C0(), S1("Km"), TIER_FP64);
  c.eng.contract(Cr(-0.5), L2("Kijb"), stable(T(c.Hovoo.c(), "mbij", {o, v, o, o})), C1(), S1("Km"),
                 tr);
  // 2h1p, one line per term of the right sigma (H_me, H_mnie, H_be, H_mi,
  // H_mnij, H_mbej, three-body), each with input and output exchanged
  c.eng.contract(C1(), L1("Ki"), T(c.Hov.c(), "me", {o, v}), C0(), G("Kime"), TIER_FP64);
  c.eng.contract(Cr(-0.5), L1("Ki"), stable(T(c.Hooov.c(), "mnie", {o, o, o, v})), C1(), G("Kmne"),
                 tr);
  c.eng.contract(Cr(0.5), L2("Kijb"), stable(T(c.Hvv_off.c(), "be", {v, v})), C1(), G("Kije"), tr);
  c.eng.contract(Cr(-1), stable(T(c.Hoo_off.c(), "mi", {o, o})), L2("Kijb"), C1(), G("Kmjb"), tr);
  c.eng.contract(Cr(0.25), L2("Kijb"), stable(T(c.Hoooo.c(), "mnij", {o, o, o, o})), C1(),
                 G("Kmnb"), tr);
  c.eng.contract(C1(), L2("Kijb"), stable(T(c.Hovvo.c(), "mbej", {o, v, v, o})), C1(), G("Kime"),
                 tr);
  c.eng.contract(Cr(0.5), L2("Kijb"), stable(T(c.t2.c(), "ijeb", {o, o, v, v})), C0(),
                 T(w.xe.c(), "Ke", {kk, v}), tr);
  c.eng.contract(Cr(-0.5), T(w.xe.c(), "Ke", {kk, v}), stable(T(c.oovv.c(), "mnef", {o, o, v, v})),
                 C1(), G("Kmnf"), tr);
  c.eng.permute_into(C1(), G("Kijb"), C0(), S2("Kijb"));
  c.eng.permute_into(Cr(-1), G("Kjib"), C1(), S2("Kijb"));
  ip_diag_apply(w.r1.c(), w.r2.c(), c.doo.c(), c.dvv.c(), kk, o, v, w.s1.c(), w.s2.c(), st);
  ip_pack(w.s1.c(), w.s2.c(), kk, o, v, sout, st);
}

}  // namespace

void batch_left_sigma(std::vector<Ctx *> &sys, const std::vector<int> &k,
                      const std::vector<const cplx *> &r, const std::vector<cplx *> &s) {
  for (size_t q = 0; q < sys.size(); ++q) {
    Ctx &c = *sys[q];
    if (!c.hbar_done) c.build_hbar();
    if (k[q] == 0) continue;
    ensure_ws(c, k[q]);
    left_sigma_body(c, k[q], r[q], s[q]);
  }
}

// ---------------------------------------------------------------------------
// block Davidson as a per-system state machine
// ---------------------------------------------------------------------------
namespace {

struct Dav {
  Ctx *c = nullptr;
  int nr = 0;
  double tol = 0;
  int max_iter = 0;
  long dim = 0;
  int max_sp = 0;
  Buf V, S, d, Xr, SX, R, G, Gm, wv, VR, Ysel, wsel, cproj, corr;
  Buf nrm;  // squared norms of new vectors / residuals, on the device
  int m = 0, it = 0, added = 0;
  enum { FULL, ADDED } pending = FULL;
  bool done = false, converged = false;
  bool isolate = false;  // stop this system alone on a non-finite residual
  int failed = 0;        // CC_ERR_* that stopped this system (0: none)
  std::vector<cplx> w_out;
  std::vector<double> rn;
  int req_k = 0;
  long req_off = 0;

  cudaStream_t st() const { return c->st; }
  void g_block(int b0, int nb, int a0, int na) {
    const long ld = max_sp;
    c->eng.contract(C1(), T(S.c() + static_cast<long>(b0) * dim, "bd", {nb, dim}),
                    conj(T(V.c() + static_cast<long>(a0) * dim, "ad", {na, dim})), C0(),
                    Tv(Gm.c() + static_cast<long>(b0) * ld + a0, "ba", {nb, na}, {ld, 1}),
                    TIER_FP64);
  }
  // orthogonalise rows vecs[0..nnew) against V[0..mbase) (two passes) and
  // among themselves; accepted rows are appended to V at mbase. Row j is
  // projected (two passes) against the rows of the block before it, which
  // already sit normalised in V, and normalised on the device; a row whose
  // norm falls below 1e-10 is zeroed in place (later projections then skip
  // it) and dropped when the block is compacted after the one read of the
  // norms at the end.
  int orth_new(cplx *vecs, int nnew, int mbase) {
    if (mbase > 0) {
      for (int pass = 0; pass < 2; ++pass) {
        c->eng.contract(C1(), T(vecs, "rd", {nnew, dim}), conj(T(V.c(), "ad", {mbase, dim})), C0(),
                        T(cproj.c(), "ra", {nnew, mbase}), TIER_FP64);
        c->eng.contract(Cr(-1), T(cproj.c(), "ra", {nnew, mbase}), T(V.c(), "ad", {mbase, dim}),
                        C1(), T(vecs, "rd", {nnew, dim}), TIER_FP64);
      }
    }
    const size_t z = sizeof(cplx);
    cplx *Vb = V.c() + static_cast<long>(mbase) * dim;
    for (int j = 0; j < nnew; ++j) {
      cplx *x = vecs + static_cast<long>(j) * dim;
      if (j > 0)
        for (int pass = 0; pass < 2; ++pass) {
          // <V_a|x> for the block's rows a < j, up to 16 per pass over x
          // (each sum split over many blocks)
          for (int a0 = 0; a0 < j; a0 += 16) {
            const int na = std::min(16, j - a0);
            const cplx *ys[16];
            for (int a = 0; a < na; ++a) ys[a] = Vb + static_cast<long>(a0 + a) * dim;
            dot_multi(ys, na, x, dim, false, cproj.c() + a0, 1, c->red.c(), 4096, st());
          }
          c->eng.contract(Cr(-1), T(cproj.c(), "ra", {1, j}), T(Vb, "ad", {j, dim}), C1(),
                          T(x, "rd", {1, dim}), TIER_FP64);
        }
      dot_dev(x, x, dim, true, nrm.c() + j, st(), c->red.c());
      normalize_or_zero(Vb + static_cast<long>(j) * dim, x, dim, nrm.c() + j, 1e-10, st());
    }
    std::vector<cplx> nh(nnew);
    d2h(nh.data(), nrm.p, z * nnew, st());
    int acc = 0;
    for (int j = 0; j < nnew; ++j) {
      if (std::sqrt(std::max(nh[j].x, 0.0)) < 1e-10) continue;
      if (acc != j)
        d2d(Vb + static_cast<long>(acc) * dim, Vb + static_cast<long>(j) * dim, z * dim, st());
      ++acc;
    }
    return acc;
  }

  void start(Ctx *ctx, int n_roots, double t, int mi) {
    c = ctx;
    nr = n_roots;
    tol = t;
    max_iter = mi;
    dim = c->dim_ip();
    max_sp = static_cast<int>(std::min<long>(dim, std::max(8 * nr, 40)));
    Allocator *al = &c->al;
    const size_t z = sizeof(cplx);
    V.reset(al, z * max_sp * dim);
    S.reset(al, z * max_sp * dim);
    d.reset(al, z * dim);
    Xr.reset(al, z * nr * dim);
    SX.reset(al, z * nr * dim);
    R.reset(al, z * nr * dim);
    corr.reset(al, z * nr * dim);
    G.reset(al, z * max_sp * max_sp);
    Gm.reset(al, z * max_sp * max_sp);
    wv.reset(al, z * max_sp);
    VR.reset(al, z * max_sp * max_sp);
    Ysel.reset(al, z * nr * max_sp);
    wsel.reset(al, z * nr);
    cproj.reset(al, z * nr * max_sp);
    nrm.reset(al, z * nr);
    w_out.assign(nr, mk(0, 0));
    rn.assign(nr, 0.0);
    ip_diag(c->Hoo.c(), c->Hvv.c(), c->o, c->v, d.c(), st());
    std::vector<cplx> dh(dim);
    d2h(dh.data(), d.p, z * dim, st());
    std::vector<long> idx(dim);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](long a, long b) { return dh[a].x < dh[b].x; });
    if (c->guess_mode > 0) {
      // first-order (optionally learned) 2h1p parts for the roots seeded at
      // a 1h element, orthonormalised into V
      std::vector<int> seeds(nr);
      for (int r = 0; r < nr; ++r) seeds[r] = idx[r] < c->o ? static_cast<int>(idx[r]) : static_cast<int>(-2 - idx[r]);
      davidson_guess(*c, seeds, corr.c());
      m = orth_new(corr.c(), nr, 0);
      if (m < nr) fail(CC_ERR_NUMERIC, "Davidson starting vectors are linearly dependent");
    } else {
      CUDA_CHECK(cudaMemsetAsync(V.p, 0, z * nr * dim, st()));
      const cplx one = mk(1.0, 0.0);
      for (int r = 0; r < nr; ++r) h2d(V.c() + r * dim + idx[r], &one, z, st());
      m = nr;
    }
    pending = FULL;
    req_k = m;
    req_off = 0;
  }

  // Called once the requested sigma vectors are in S[req_off ..].
  void step() {
    if (pending == FULL) {
      g_block(0, m, 0, m);
    } else {
      g_block(m, added, 0, m + added);  // new columns
      g_block(0, m, m, added);          // new rows
      m += added;
    }
    ++it;
    const size_t z = sizeof(cplx);
    const long ld = max_sp;
    c->eng.permute_into(C1(), Tv(Gm.c(), "ba", {m, m}, {ld, 1}), C0(), T(G.c(), "ba", {m, m}));
    {
      // a non-finite subspace matrix (a NaN or Inf sigma) stops this system
      // before the eigensolver sees it
      std::vector<cplx> gh(static_cast<size_t>(m) * m);
      d2h(gh.data(), G.p, z * m * m, st());
      for (const cplx &x : gh)
        if (!std::isfinite(x.x) || !std::isfinite(x.y)) {
          if (!isolate) fail(CC_ERR_NUMERIC, "Davidson subspace matrix is not finite");
          failed = CC_ERR_NUMERIC;
          done = true;
          return;
        }
    }
    geev_dev(&c->al, st(), G.c(), m, wv.c(), VR.c());
    std::vector<cplx> wh(m), vh(static_cast<size_t>(m) * m);
    CUDA_CHECK(cudaMemcpyAsync(wh.data(), wv.p, z * m, cudaMemcpyDeviceToHost, st()));
    d2h(vh.data(), VR.p, z * m * m, st());  // one synchronisation for both
    std::vector<int> ord(m);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return wh[a].x < wh[b].x; });
    std::vector<cplx> ys(static_cast<size_t>(nr) * m);
    for (int r = 0; r < nr; ++r) {
      const int col = ord[r];
      double nn = 0;
      for (int a = 0; a < m; ++a)
        nn += vh[col * m + a].x * vh[col * m + a].x + vh[col * m + a].y * vh[col * m + a].y;
      nn = 1.0 / std::sqrt(nn);
      for (int a = 0; a < m; ++a) ys[r * m + a] = cscale(nn, vh[col * m + a]);
      w_out[r] = wh[col];
    }
    h2d(Ysel.p, ys.data(), z * nr * m, st());
    h2d(wsel.p, w_out.data(), z * nr, st());
    c->eng.contract(C1(), T(Ysel.c(), "ra", {nr, m}), T(V.c(), "ad", {m, dim}), C0(),
                    T(Xr.c(), "rd", {nr, dim}), TIER_FP64);
    c->eng.contract(C1(), T(Ysel.c(), "ra", {nr, m}), T(S.c(), "ad", {m, dim}), C0(),
                    T(SX.c(), "rd", {nr, dim}), TIER_FP64);
    d2d(R.p, SX.p, z * nr * dim, st());
    for (int r = 0; r < nr; ++r) {
      axpby(dim, mk(-w_out[r].x, -w_out[r].y), Xr.c() + r * dim, C1(), R.c() + r * dim, st());
      dot_dev(R.c() + r * dim, R.c() + r * dim, dim, true, nrm.c() + r, st(), c->red.c());
    }
    std::vector<cplx> n2h(nr);
    d2h(n2h.data(), nrm.p, z * nr, st());
    bool all = true;
    for (int r = 0; r < nr; ++r) {
      rn[r] = std::sqrt(std::max(n2h[r].x, 0.0));
      if (!std::isfinite(rn[r])) {
        if (!isolate) fail(CC_ERR_NUMERIC, "Davidson residual NaN");
        failed = CC_ERR_NUMERIC;
        done = true;
        return;
      }
      if (rn[r] >= tol) all = false;
    }
    if (all) {
      converged = done = true;
      return;
    }
    if (it >= max_iter) {
      done = true;
      return;
    }
    std::vector<int> todo;
    for (int r = 0; r < nr; ++r)
      if (rn[r] >= tol) todo.push_back(r);
    if (m + static_cast<int>(todo.size()) > max_sp) {
      // restart from the Ritz vectors
      d2d(corr.p, Xr.p, z * nr * dim, st());
      m = orth_new(corr.c(), nr, 0);
      pending = FULL;
      req_k = m;
      req_off = 0;
      return;
    }
    precondition(R.c(), wsel.c(), d.c(), nr, dim, SX.c(), st());  // SX as scratch
    for (size_t j = 0; j < todo.size(); ++j)
      d2d(corr.c() + j * dim, SX.c() + static_cast<long>(todo[j]) * dim, z * dim, st());
    added = orth_new(corr.c(), static_cast<int>(todo.size()), m);
    if (added == 0) {
      done = true;
      return;
    }
    pending = ADDED;
    req_k = added;
    req_off = m;
  }

  void results(double *omega, double *r1w) {
    if (!c) {  // never started: no roots
      for (int r = 0; r < nr; ++r) {
        omega[2 * r] = omega[2 * r + 1] = 0.0;
        if (r1w) r1w[r] = 0.0;
      }
      return;
    }
    for (int r = 0; r < nr; ++r) {
      omega[2 * r] = w_out[r].x;
      omega[2 * r + 1] = w_out[r].y;
      if (r1w) {
        const cplx a = dot(Xr.c() + r * dim, Xr.c() + r * dim, c->o, true, st(), c->red.c());
        const cplx b = dot(Xr.c() + r * dim, Xr.c() + r * dim, dim, true, st(), c->red.c());
        r1w[r] = a.x / b.x;
      }
    }
  }
};

}  // namespace

// Lockstep block Davidson over several systems (one batched sigma per round).
// status[q] = CC_OK or CC_ERR_NOT_CONVERGED per system (and, with isolate,
// the error that stopped that system alone).
void run_ipeom(std::vector<Ctx *> &sys, int nr, double tol, int max_iter, double *omega,
               double *r1w, int *n_iter, int *status, bool use_graph, bool left,
               const std::vector<cplx *> *vecs, bool isolate) {
  const double t0 = now_ms();
  std::vector<Dav> dv(sys.size());
  for (size_t q = 0; q < sys.size(); ++q) {
    Ctx *c = sys[q];
    dv[q].nr = nr;
    dv[q].isolate = isolate;
    try {
      if (!c->ccsd_done) fail(CC_ERR_STATE, "ipeom needs a converged ccsd_solve");
      if (nr < 1 || nr > c->dim_ip() || nr > 64) fail(CC_ERR_ARG, "n_roots out of range");
      if (!c->hbar_done) c->build_hbar();
      dv[q].start(c, nr, tol, max_iter);
    } catch (const Error &e) {
      if (!isolate) throw;
      c->last_error = e.msg;
      dv[q] = Dav();
      dv[q].nr = nr;
      dv[q].failed = e.code;
      dv[q].done = true;
    }
  }
  while (true) {
    std::vector<Ctx *> act;
    std::vector<int> ks;
    std::vector<const cplx *> rs;
    std::vector<cplx *> ss;
    std::vector<Dav *> ad;
    for (auto &d : dv) {
      if (d.done) continue;
      act.push_back(d.c);
      ks.push_back(d.req_k);
      rs.push_back(d.V.c() + d.req_off * d.dim);
      ss.push_back(d.S.c() + d.req_off * d.dim);
      ad.push_back(&d);
    }
    if (act.empty()) break;
    if (left)
      batch_left_sigma(act, ks, rs, ss);
    else
      batch_sigma(act, ks, rs, ss, use_graph);
    for (Dav *d : ad) d->c->maybe_inject(2, d->it + 1, d->S.c() + d->req_off * d->dim);
    for (auto &d : dv) {
      if (d.done) continue;
      if (!isolate) {
        d.step();
        continue;
      }
      try {
        d.step();
      } catch (const Error &e) {
        if (e.code == CC_ERR_CUDA || e.code == CC_ERR_OOM || e.code == CC_ERR_TIMEOUT) throw;
        d.c->last_error = e.msg;
        d.failed = e.code;
        d.done = true;
      }
    }
  }
  for (size_t q = 0; q < sys.size(); ++q) {
    dv[q].results(omega + 2L * nr * q, r1w ? r1w + static_cast<long>(nr) * q : nullptr);
    if (n_iter) n_iter[q] = dv[q].it;
    if (status)
      status[q] = dv[q].failed ? dv[q].failed : (dv[q].converged ? CC_OK : CC_ERR_NOT_CONVERGED);
    if (!dv[q].c) continue;
    if (vecs) d2d((*vecs)[q], dv[q].Xr.p, sizeof(cplx) * nr * dv[q].dim, dv[q].st());
    sys[q]->stat[8] = dv[q].it;
    sys[q]->check_err_flag();
  }
  const double dt = now_ms() - t0;
  for (Ctx *c : sys) c->stat[5] += dt / sys.size();
  for (Ctx *c : sys) c->settle_sigma_timing();
  for (Ctx *c : sys) c->eng.trace_flush();
}

}  // namespace cdfns
