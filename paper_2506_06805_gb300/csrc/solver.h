// Solver state of one system and the host orchestration of the hot path.
#pragma once

#include <memory>
#include <string>
#include <vector>

#include "cc_kernels.h"
#include "engine.h"

namespace cdfns {

struct Ctx {
  int o = 0, v = 0, X = 0;  // current occupied / virtual / auxiliary sizes
  int v_input = 0;          // virtual count given at init (before FNS)
  std::vector<double> eps;  // host copy, occupied first
  Allocator al;
  cudaStream_t st = nullptr;
  Engine eng;
  int tier = TIER_FP64;
  int eom_tier = -1;  // -1: same as tier
  bool use_graphs = true;  // replay the batched sigma from CUDA graphs
  int num_sms = 148;
  size_t slab_budget = size_t(4) << 30;  // bytes for ladder V slabs
  int diis_depth = 0;                    // DIIS pairs held in the last ccsd_solve
  int cc_tier = -1;       // tier of the CCSD residual while ccsd_solve runs (-1: tier)
  int cc_done_tier = -1;  // tier the last ccsd_solve finished in (-1: none)

  // inputs
  Buf eps_d;
  Buf Loo, Lov, Lvo, Lvv;  // [X][o][o], [X][o][v], [X][v][o], [X][v][v]
  std::vector<char> have_P;
  long n_have = 0;
  bool input_checked = false;
  Buf stats_d, err_d, red;

  // stored integrals (at most two virtual indices)
  bool ints = false;
  Buf oooo, ooov, oovv, ovvo;
  Buf ovvo_jbme;  // <mb||ej> as [j][b][m][e], held during ccsd_solve

  // amplitudes
  Buf t1, t2;
  bool amps = false, amps_user = false, ccsd_done = false, fns_done = false;
  cplx e_corr = {0, 0};

  // H-bar
  bool hbar_done = false;
  Buf Hov, Hoo, Hvv, Hoooo, Hooov, Hovvo, Hovoo;
  Buf Hoo_off, Hvv_off, doo, dvv;  // one-body H-bar split into diagonal + rest

  // pair tables (row-major i<j over o, a<b over v)
  Buf ij_i, ij_j, ab_a, ab_b;
  int pairs_o = -1, pairs_v = -1;

  // persistent workspace of the batched sigma (kept for CUDA-graph replay)
  struct SigmaWS {
    long kcap = 0;
    Buf rin, sout, r1, r2, s1, s2, tA, tB, tC, X1, X2, xe;
  } sws;
  long sig_gen = 0;  // bumped whenever H-bar or the sigma workspace changes

  std::vector<double> fns_occ;
  // streamed natural spinors (cc_begin_fns_stream): 0 off, 1 first pass
  // over the Cholesky chunks (occupied blocks kept, L_vv dropped), 2 second
  // pass (each chunk's L_vv rotated into the kept basis), 3 done
  int fns_stream = 0;
  Buf U_fns, Lvv_kept;        // rotation [v][nk] and the rotated L_vv [X][nk][nk]
  std::vector<double> eps_kept;
  std::vector<char> have_P2;
  long n_have2 = 0;
  double fns_ms = 0;
  double stat[24] = {0};
  // CUDA events around each batched sigma build this context took part in,
  // shared by the systems of that batch (destroyed with the last reference)
  struct EventPair {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~EventPair() {
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
    }
  };
  std::vector<std::shared_ptr<EventPair>> sig_timing;
  // CUDA events around each ladder call, read when the calling solve ends
  // (no synchronisation in the middle of a residual)
  std::vector<std::shared_ptr<EventPair>> ladder_timing;
  // adds the device time of the recorded ladder calls to stat[0] and their
  // count to stat[1], and releases the events
  void settle_ladder_timing();
  // adds the device time of the recorded sigma builds to stat[16], their
  // count to stat[17], and releases the events
  void settle_sigma_timing();
  std::string last_error;
  // Davidson start (cc_set_davidson_guess): 0 unit vectors at the lowest
  // diagonal elements, 1 first-order 2h1p components for 1h-seeded roots,
  // 2 the same scaled by the network guess_mlp (a cc_mlp's state)
  int guess_mode = 0;
  const void *guess_mlp = nullptr;
  // right vectors of the last ipeom_solve ([last_nr][dim], unit norm)
  Buf last_R;
  int last_nr = 0;
  // host-side fault injection for tests of the error paths
  // (cc_set_fault_injection): kind 1 writes NaN into the CCSD residual of
  // iteration `inject_at`, kind 2 into the sigma vectors of Davidson
  // iteration `inject_at`; cleared once it has fired
  int inject_kind = 0, inject_at = 0;
  void maybe_inject(int kind, int iteration, cplx *target);

  // --- lifecycle ---
  void create(int n_occ, int n_virt, int n_aux, const double *eps_host);
  // L chunk [p1-p0][n][n] complex128 in host memory, or device memory (on_device)
  void add_chunk(int p0, int p1, const double *L, bool on_device = false);
  void validate_input();
  void ensure_ready();
  void build_integrals();
  // --- solvers ---
  int fns(double threshold, int n_keep);
  void begin_fns_stream();
  int fns_stream_truncate(double threshold, int n_keep);
  void rotate_chunk(int p0, int p1, const double *L, bool on_device);
  void finish_fns_stream();
  int ccsd(double tol, int max_iter, double *e_out, int *n_iter);
  int ipeom(int n_roots, double tol, int max_iter, double *omega, double *r1w, int *n_iter);
  // right and left vectors (Eqs. 18-20), biorthonormal: L^T R = 1
  int ipeom_lr(int n_roots, double tol, int max_iter, double *omega, cplx *R_dev, cplx *L_dev,
               int *n_iter);
  // --- components ---
  void residual(const cplx *t1, const cplx *t2, cplx *R1, cplx *R2);
  // tau_amax (FP16 tiers, optional): a device float >= max |tau| (FP32 of
  // |Re|, |Im|) over the whole tensor
  void ladder(const cplx *Lv, const cplx *tau, cplx *R2, int tier, const float *tau_amax = nullptr);
  void build_hbar();
  void sigma(int k, const cplx *r, cplx *s);
  void left_sigma(int k, const cplx *l, cplx *s);
  cplx energy(const cplx *t1, const cplx *t2);
  void check_err_flag();
  void ensure_pairs();
  // upper estimate of the scratch planes of the tensor-core operands
  size_t planes_bytes_estimate(int tier) const;
  // upper estimate of the device bytes one CCSD residual allocates and frees
  // again (tau, tau~, X, W, z, the dressed L, ladder slabs, operand planes)
  size_t residual_bytes_estimate() const;
  int eom() const { return eom_tier < 0 ? tier : eom_tier; }
  // integrals and FNS: the accurate split tier of the chosen family
  int int_tier() const { return tier_accurate(tier); }
  // H-bar is built once from the CCSD amplitudes with the residual's kinds
  // of contractions, in the tier the CCSD iterations finished in (FP16 H-bar
  // moves the IPs of the small workload by 3e-9 Eh from FP64); the Davidson
  // sigma uses the EOM tier
  int hbar_tier() const { return cc_done_tier >= 0 ? cc_done_tier : tier; }
  int res_tier() const { return cc_tier >= 0 ? cc_tier : tier; }
  long nij() const { return static_cast<long>(o) * (o - 1) / 2; }
  long nab() const { return static_cast<long>(v) * (v - 1) / 2; }
  long dim_ip() const { return o + nij() * v; }
  long n_amp() const { return static_cast<long>(o) * v + nij() * nab(); }
  cplx *B(Buf &b, size_t n) {  // (re)allocate n complex elements
    if (b.bytes < n * sizeof(cplx)) b.reset(&al, n * sizeof(cplx));
    return b.c();
  }
};

// eom.cu: batched sigma, lockstep block Davidson, graph cache
void batch_sigma(std::vector<Ctx *> &sys, const std::vector<int> &k,
                 const std::vector<const cplx *> &r, const std::vector<cplx *> &s, bool use_graph);
// Lockstep block Davidson; `left` solves l^T H-bar = omega l^T instead
// (transposed sigma, no graphs); `vecs` (device, per system) receives the
// nr Ritz vectors [nr][dim] when given.
// With isolate, a system that cannot start (no converged CCSD, n_roots out
// of range) or whose iteration turns non-finite stops with its own status
// (CC_ERR_STATE, CC_ERR_ARG, CC_ERR_NUMERIC) while the others go on;
// without it such a failure is raised for the whole call.
void run_ipeom(std::vector<Ctx *> &sys, int nr, double tol, int max_iter, double *omega,
               double *r1w, int *n_iter, int *status, bool use_graph, bool left = false,
               const std::vector<cplx *> *vecs = nullptr, bool isolate = false);
void batch_left_sigma(std::vector<Ctx *> &sys, const std::vector<int> &k,
                      const std::vector<const cplx *> &r, const std::vector<cplx *> &s);
void drop_graphs(const void *ctx);
// mlp.cu: starting vectors V [seeds.size()][dim] of the Davidson iterations
// for c.guess_mode 1 or 2; seeds[r] >= 0 is the 1h element root r is seeded
// at, -2 - pos a root that starts as the unit vector at 2h1p position pos.
void davidson_guess(Ctx &c, const std::vector<int> &seeds, cplx *V);
void geev_dev(Allocator *al, cudaStream_t st, cplx *A, int m, cplx *w, cplx *vr);

}  // namespace cdfns

// The opaque handle of the C ABI wraps one solver state.
struct cc_ctx {
  cdfns::Ctx c;
};
