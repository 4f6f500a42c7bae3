// C ABI of the discloop library: context, gauge loading, noise, operators,
// the batched mixed-precision CG with reliable updates, contractions and the
// Truncated Solver Method driver.  Every arithmetic step runs in the kernels of
// dl_dslash.cu, dl_blas.cu, dl_layout.cu and dl_contract.cu; this file only
// orders launches, owns device memory and reads back per-column scalars.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <map>
#include <string>
#include <vector>

#include "discloop.h"
#include "dl_host.h"

#include <atomic>
#include <mutex>

static std::atomic<long long> g_launches{0};
void dl_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }


namespace dlh {

dl_status fail(dl_ctx* c, dl_status s, const std::string& m) {
  if (c) c->err = m;
  return s;
}

dl_status cuda_fail(dl_ctx* c, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  if (c) c->err = m;
  return e == cudaErrorMemoryAllocation ? DL_ERR_OOM : DL_ERR_CUDA;
}


Batch make_batch(const dl_ctx* c, int ncol) {
  Batch B;
  memset(&B, 0, sizeof(B));
  B.nlat = 1;
  LatDesc& L = B.lat[0];
  L.X = c->dims[0];
  L.Y = c->dims[1];
  L.Z = c->dims[2];
  L.T = c->dims[3];
  L.Vh = c->Vh;
  L.lognpad = ilog2ceil(std::max(ncol, 1));
  L.ncol = ncol;
  L.rhs_base = 0;
  L.item_off = 0;
  L.gsite_off = 0;
  L.tbc = c->lats[0].tbc;
  L.kappa = c->lats[0].kappa;
  L.amu = c->lats[0].amu;
  L.noise_base = 0;
  B.pstride = (int)c->partial_blocks;
  dl::blocks_for(B, 256);
  return B;
}

// Batch over every lattice of the context: each lattice's n columns are split
// into instances of `tile` columns (the last one ragged) sharing its gauge field;
// instance k of lattice l draws noise indices l * n + k * tile + column.
bool make_batch_multi(const dl_ctx* c, int tile, int n, Batch& B) {
  memset(&B, 0, sizeof(B));
  long long item = 0;
  int rhs = 0;
  for (int l = 0; l < (int)c->lats.size(); ++l) {
    const LatInfo& LI = c->lats[l];
    for (int k = 0; k * tile < n; ++k) {
      if (B.nlat >= DL_MAX_LAT) return false;
      LatDesc& L = B.lat[B.nlat++];
      L.X = LI.dims[0];
      L.Y = LI.dims[1];
      L.Z = LI.dims[2];
      L.T = LI.dims[3];
      L.Vh = LI.Vh;
      L.lognpad = ilog2ceil(tile);
      L.ncol = std::min(tile, n - k * tile);
      L.rhs_base = rhs;
      L.item_off = item;
      L.gsite_off = LI.gsite_off;
      L.tbc = LI.tbc;
      L.kappa = LI.kappa;
      L.amu = LI.amu;
      L.noise_base = (long long)l * n + (long long)k * tile;
      rhs += L.ncol;
      item += (long long)L.Vh << L.lognpad;
    }
  }
  if (rhs > DL_NCMAX) return false;
  B.pstride = (int)c->partial_blocks;
  // more than 32 padded columns per lattice would overrun the partial-sum buffer
  return (size_t)dl::blocks_for(B, 256) <= c->partial_blocks;
}

// Site factor T = a + i b gamma_5 of R_f (inv = false) or R_f^{-1} (inv = true) for
// one lattice's kappa and a*mu.
void twist_ab_l(const LatDesc& L, int f, bool inv, double& a, double& b) {
  double w = 2.0 * L.kappa * L.amu * f;
  if (!inv) {
    a = 1.0;
    b = w;
  } else {
    a = 1.0 / (1.0 + w * w);
    b = -w / (1.0 + w * w);
  }
}

// Epilogue coefficient kinds, evaluated per lattice of a batch.

// kinds of site factor: 0 identity, 1 R_f, 2 R_f^{-1}; every lattice of B gets its own
EpiSet epiB(const Batch& B, int ck, int t1, int f1, int t2, int f2) {
  EpiSet E;
  memset(&E, 0, sizeof(E));
  for (int l = 0; l < B.nlat; ++l) {
    const LatDesc& L = B.lat[l];
    Epi& e = E.e[l];
    e.c = ck == CK_ONE ? 1.0 : (ck == CK_K ? L.kappa : (ck == CK_MK ? -L.kappa : -L.kappa * L.kappa));
    e.a1 = 1.0;
    e.b1 = 0.0;
    e.a2 = 1.0;
    e.b2 = 0.0;
    if (t1) twist_ab_l(L, f1, t1 == 2, e.a1, e.b1);
    if (t2) twist_ab_l(L, f2, t2 == 2, e.a2, e.b2);
    auto split = [](double v, float& f, float& l) {
      f = (float)v;
      l = (float)(v - (double)f);
    };
    split(e.c, e.cf, e.cl);
    split(e.a1, e.a1f, e.a1l);
    split(e.b1, e.b1f, e.b1l);
    split(e.a2, e.a2f, e.a2l);
    split(e.b2, e.b2f, e.b2l);
  }
  return E;
}

int ncols_of(const Batch& B) {
  int n = 0;
  for (int l = 0; l < B.nlat; ++l) n += B.lat[l].ncol;
  return n;
}

size_t items_of(const Batch& B) {
  size_t n = 0;
  for (int l = 0; l < B.nlat; ++l) n += (size_t)B.lat[l].Vh << B.lat[l].lognpad;
  return n;
}

int grec_of(const dl_ctx* c, int prec) {
  return (prec == P64 || prec == PDF) ? 18 : (prec == P32 ? c->rec32 : c->rec16);
}

void invalidate_graphs(dl_ctx* c) {
  for (auto& g : c->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
}

dl_status ensure_field(dl_ctx* c, const std::string& base, int prec, const Batch& B, Field** out) {
  const size_t items = items_of(B);
  const std::string name = base + "#" + std::to_string(prec);
  auto it = c->ws.find(name);
  if (it != c->ws.end() && it->second.prec == prec && it->second.items >= items) {
    *out = &it->second;
    return DL_OK;
  }
  if (it != c->ws.end()) {
    cudaFree(it->second.data);
    if (it->second.norm) cudaFree(it->second.norm);
    c->ws.erase(it);
    invalidate_graphs(c);
  }
  Field f;
  f.prec = prec;
  f.items = items;
  CK(cudaMalloc(&f.data, items * chunk_bytes(prec)));
  if (prec == P16) CK(cudaMalloc((void**)&f.norm, items * sizeof(float)));
  c->ws[name] = f;
  *out = &c->ws[name];
  return DL_OK;
}

// The partial-sum buffer holds DL_MAXC columns of pstride blocks, enough for any
// launch on this context (256-thread blocks over Vh * 32 items); allocated once.
dl_status ensure_partial(dl_ctx* c, const Batch& B) {
  size_t nb = (size_t)B.blk_begin[B.nlat];
  if (nb <= c->partial_blocks) return DL_OK;
  return fail(c, DL_ERR_STATE, "partial-sum buffer smaller than a launch");
}

dl_status ensure_scratch(dl_ctx* c, size_t bytes) {
  if (bytes <= c->scratch_bytes) return DL_OK;
  if (c->scratch) cudaFree(c->scratch);
  c->scratch = nullptr;
  c->scratch_bytes = 0;
  CK(cudaMalloc(&c->scratch, bytes));
  c->scratch_bytes = bytes;
  return DL_OK;
}

dl_status ensure_buf(dl_ctx* c, const std::string& name, size_t bytes, void** out) {
  auto it = c->bufs.find(name);
  if (it != c->bufs.end() && it->second.bytes >= bytes) {
    *out = it->second.p;
    return DL_OK;
  }
  if (it != c->bufs.end()) {
    cudaFree(it->second.p);
    c->bufs.erase(it);
  }
  DevBuf b;
  CK(cudaMalloc(&b.p, std::max<size_t>(bytes, 16)));
  b.bytes = bytes;
  c->bufs[name] = b;
  *out = b.p;
  return DL_OK;
}

// entry/exit ordering against the caller's stream
dl_status enter(dl_ctx* c) {
  CK(cudaSetDevice(c->dev));
  CK(cudaEventRecord(c->ev_in, c->user));
  CK(cudaStreamWaitEvent(c->st, c->ev_in, 0));
  return DL_OK;
}
dl_status leave(dl_ctx* c) {
  CK(cudaEventRecord(c->ev_out, c->st));
  CK(cudaStreamWaitEvent(c->user, c->ev_out, 0));
  return DL_OK;
}

const FieldRef NOF = {nullptr, nullptr};

// ---- operator stages (even-odd, App. A Eq. A.2) ----------------------------
// out_o = R_{f'}^{-1} D^{(dag)}_oe in_e,  f' = dag ? -f : f
cudaError_t stage1(dl_ctx* c, const Batch& B, int prec, bool dag, int f, FieldRef in_e, FieldRef out_o, const int* mask) {
  int ff = dag ? -f : f;
  EpiSet E = epiB(B, CK_ONE, 2, ff, 0, 0);
  GaugeSet g{c->g64, c->g32, c->g16, c->gdf};
  return dl::dslash(B, prec, grec_of(c, prec), EPI_PLAIN, dag, 1, in_e, NOF, out_o, g, E, mask, nullptr, NOF, NOF, NOF,
                    nullptr, c->st);
}
// out_e = R_{f'} aux_e - kappa^2 D^{(dag)}_eo in_o  (optionally |out|^2 partials)
cudaError_t stage2(dl_ctx* c, const Batch& B, int prec, bool dag, int f, FieldRef in_o, FieldRef aux_e, FieldRef out_e,
                   const int* mask, double* partial) {
  int ff = dag ? -f : f;
  EpiSet E = epiB(B, CK_MK2, 0, 0, 1, ff);
  GaugeSet g{c->g64, c->g32, c->g16, c->gdf};
  return dl::dslash(B, prec, grec_of(c, prec), partial ? EPI_AUX_NORM : EPI_AUX, dag, 0, in_o, aux_e, out_e, g, E, mask,
                    partial, NOF, NOF, NOF, nullptr, c->st);
}

// Ax = Mhat^dag Mhat x (all in one precision), using two temporaries
cudaError_t normal_op(dl_ctx* c, const Batch& B, int prec, int f, FieldRef x, FieldRef t_o, FieldRef q_e, FieldRef t2_o,
                      FieldRef ax, const int* mask) {
  DL_CUDA_TRY(stage1(c, B, prec, false, f, x, t_o, mask));
  DL_CUDA_TRY(stage2(c, B, prec, false, f, t_o, x, q_e, mask, nullptr));
  DL_CUDA_TRY(stage1(c, B, prec, true, f, q_e, t2_o, mask));
  return stage2(c, B, prec, true, f, t2_o, q_e, ax, mask, nullptr);
}

// per-column sums of the partial buffer into S[slot]
cudaError_t colsum(dl_ctx* c, const Batch& B, int slot) {
  return dl::sum_partials(B, c->partial, c->S, DL_NCMAX, slot, ncols_of(B), c->st);
}

// ---- the CG on the normal equations ----------------------------------------
struct CGState {
  std::vector<double> S;
  std::vector<int> active, flags, iters;
};

dl_status download_state(dl_ctx* c, int n, CGState& h) {
  h.S.resize(DL_NS * DL_NCMAX);
  h.active.resize(n);
  h.flags.resize(n);
  h.iters.resize(n);
  CK(cudaMemcpyAsync(h.S.data(), c->S, sizeof(double) * DL_NS * DL_NCMAX, cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(h.active.data(), c->active, sizeof(int) * n, cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(h.flags.data(), c->flags, sizeof(int) * n, cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(h.iters.data(), c->iters, sizeof(int) * n, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  return DL_OK;
}

dl_status upload_state(dl_ctx* c, int n, const CGState& h) {
  CK(cudaMemcpyAsync(c->S, h.S.data(), sizeof(double) * DL_NS * DL_NCMAX, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->active, h.active.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->flags, h.flags.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  return DL_OK;
}

struct CGFields {
  Field *r, *p, *y, *t1, *q, *t2;      // low precision
  Field *rh, *ax, *th1, *tq, *th2;     // high precision temporaries
};

// One CG iteration for all active columns (low precision); graph-capturable.
cudaError_t cg_iteration(dl_ctx* c, const Batch& B, int lo, int f, const CGFields& F, double tol2, double delta) {
  const int n = ncols_of(B);
  DL_CUDA_TRY(stage1(c, B, lo, false, f, F.p->ref(), F.t1->ref(), c->active));
  DL_CUDA_TRY(stage2(c, B, lo, false, f, F.t1->ref(), F.p->ref(), F.q->ref(), c->active, c->partial));
  DL_CUDA_TRY(colsum(c, B, DL_S_PAP));
  DL_CUDA_TRY(dl::cg_alpha(n, c->S, c->active, c->flags, c->st));
  DL_CUDA_TRY(stage1(c, B, lo, true, f, F.q->ref(), F.t2->ref(), c->active));
  {
    EpiSet E = epiB(B, CK_MK2, 0, 0, 1, -f);
    GaugeSet g{c->g64, c->g32, c->g16, c->gdf};
    DL_CUDA_TRY(dl::dslash(B, lo, grec_of(c, lo), EPI_CG, true, 0, F.t2->ref(), F.q->ref(), NOF, g, E, c->active,
                           c->partial, F.r->ref(), F.y->ref(), F.p->ref(), c->S + DL_S_ALPHA * DL_NCMAX, c->st));
  }
  DL_CUDA_TRY(colsum(c, B, DL_S_RRNEW));
  DL_CUDA_TRY(dl::cg_beta(n, c->S, c->active, c->flags, c->iters, tol2, delta, c->st));
  return dl::xpay(B, lo, F.p->ref(), F.r->ref(), c->S + DL_S_BETA * DL_NCMAX, c->active, c->st);
}

// One timed application of the four stencil stages of an iteration (all columns,
// outside the solver's graph) on the solver's current fields; used by dl_profile.
// Runs after a solve has finished: it leaves r and y modified, which the next
// solve re-initialises.
dl_status sample_stencil(dl_ctx* c, const Batch& B, int lo, int f, const CGFields& F) {
  struct Sampling {  // these launches are extra profiling work: timed, not counted
    Sampling() { dl::stencil_prof_sampling(true); }
    ~Sampling() { dl::stencil_prof_sampling(false); }
  } sampling;
  GaugeSet g{c->g64, c->g32, c->g16, c->gdf};
  cudaEvent_t* ev = c->pev;
  CK(cudaEventRecord(ev[0], c->st));
  CK(stage1(c, B, lo, false, f, F.p->ref(), F.t1->ref(), nullptr));
  CK(cudaEventRecord(ev[1], c->st));
  CK(cudaEventRecord(ev[2], c->st));
  CK(stage2(c, B, lo, false, f, F.t1->ref(), F.p->ref(), F.q->ref(), nullptr, c->partial));
  CK(cudaEventRecord(ev[3], c->st));
  CK(cudaEventRecord(ev[4], c->st));
  CK(stage1(c, B, lo, true, f, F.q->ref(), F.t2->ref(), nullptr));
  CK(cudaEventRecord(ev[5], c->st));
  EpiSet E = epiB(B, CK_MK2, 0, 0, 1, -f);
  CK(cudaEventRecord(ev[6], c->st));
  CK(dl::dslash(B, lo, grec_of(c, lo), EPI_CG, true, 0, F.t2->ref(), F.q->ref(), NOF, g, E, nullptr, c->partial,
                F.r->ref(), F.y->ref(), F.p->ref(), c->S + DL_S_ALPHA * DL_NCMAX, c->st));
  CK(cudaEventRecord(ev[7], c->st));
  CK(cudaStreamSynchronize(c->st));
  for (int k = 0; k < 4; ++k) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]));
    const int slot = lo == PDF ? P64 : lo;
    c->prof_ms[k][slot] += ms;
    c->prof_n[k][slot] += 1;
    long long it = 0;
    for (int l = 0; l < B.nlat; ++l) it += (long long)B.lat[l].Vh * B.lat[l].ncol;
    c->prof_items[k][slot] += it;  // site-column items with every column active
  }
  return DL_OK;
}

// Reliable update for the columns in `mask` (host vector): x += y, y = 0,
// r_hi = b - A x (high precision), r = r_hi.  Returns |r_hi|^2 per column.
dl_status reliable_update(dl_ctx* c, const Batch& B, int hi, int lo, int f, const CGFields& F, Field* x, Field* b,
                          const std::vector<int>& mask, std::vector<double>& rr_true) {
  const int n = ncols_of(B);
  CK(cudaMemcpyAsync(c->upd, mask.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c->st));
  CK(dl::accum(B, hi, lo, x->ref(), F.y->ref(), c->upd, 1, c->st));
  CK(normal_op(c, B, hi, f, x->ref(), F.th1->ref(), F.tq->ref(), F.th2->ref(), F.ax->ref(), c->upd));
  CK(dl::xmy_norm(B, hi, F.rh->ref(), b->ref(), F.ax->ref(), c->upd, c->partial, c->st));
  CK(colsum(c, B, DL_S_TMP));
  CK(dl::copy(B, lo, hi, F.r->ref(), F.rh->ref(), c->upd, c->st));
  std::vector<double> S(DL_NS * DL_NCMAX);
  CK(cudaMemcpyAsync(S.data(), c->S, sizeof(double) * DL_NS * DL_NCMAX, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  rr_true.assign(n, 0.0);
  for (int i = 0; i < n; ++i) rr_true[i] = S[DL_S_TMP * DL_NCMAX + i];
  return DL_OK;
}

std::string graph_key(const dl_ctx* c, const Batch& B, int lo, int f, double tol2, double delta, const CGFields& F) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%d|%d|%.17g|%.17g|%p|%p|%p|%p|%p|%p|%p|%d|%d|", lo, f, tol2, delta, F.r->data, F.p->data,
           F.y->data, F.t1->data, F.q->data, F.t2->data, (void*)c->partial, c->rec32, c->rec16);
  std::string k(buf);
  for (int l = 0; l < B.nlat; ++l) {
    const LatDesc& L = B.lat[l];
    snprintf(buf, sizeof(buf), "%d.%d.%d.%d.%d.%d.%lld.%lld.%.17g.%.17g.%.17g;", L.X, L.Y, L.Z, L.T, L.lognpad, L.ncol,
             L.item_off, L.gsite_off, L.kappa, L.amu, L.tbc);
    k += buf;
  }
  return k;
}

// The solver's graph: a conditional WHILE node whose body is one CG iteration
// followed by cg_cond, which stops the loop on the device as soon as no column
// is active, a column waits for a reliable update, or the launch's iteration
// limit (loopctr[1]) is reached.  One launch runs as many iterations as needed.
dl_status get_graph(dl_ctx* c, const Batch& B, int lo, int f, const CGFields& F, double tol2, double delta,
                    GraphEntry** out) {
  std::string key = graph_key(c, B, lo, f, tol2, delta, F);
  for (auto& g : c->graphs)
    if (g.key == key) {
      *out = &g;
      return DL_OK;
    }
  cudaGraph_t outer;
  CK(cudaGraphCreate(&outer, 0));
  cudaGraphConditionalHandle h;
  CK(cudaGraphConditionalHandleCreate(&h, outer, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, outer, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  const long long before = g_launches.load();
  CK(cudaStreamBeginCaptureToGraph(c->st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  dl::stencil_capture_begin();
  cudaError_t e = cg_iteration(c, B, lo, f, F, tol2, delta);
  if (e == cudaSuccess)
    e = dl::cg_cond(ncols_of(B), c->active, c->flags, c->loopctr, c->loopctr + 1, c->waitc, h, nullptr, c->st);
  const dl::StencilTally tally = dl::stencil_capture_end();
  cudaGraph_t captured;
  cudaError_t e2 = cudaStreamEndCapture(c->st, &captured);
  if (e != cudaSuccess) {
    cudaGraphDestroy(outer);
    return cuda_fail(c, e, "capture of the CG iteration");
  }
  CK(e2);
  cudaGraphExec_t exec;
  CK(cudaGraphInstantiate(&exec, outer, 0));
  cudaGraphDestroy(outer);
  const long long nodes = g_launches.load() - before;
  g_launches.fetch_sub(nodes);  // counted per executed iteration, not at capture
  if (c->graphs.size() >= 8) {
    cudaGraphExecDestroy(c->graphs.front().exec);
    c->graphs.erase(c->graphs.begin());
  }
  c->graphs.push_back(GraphEntry{key, exec, nodes, tally});
  *out = &c->graphs.back();
  return DL_OK;
}

// Solve Mhat^dag Mhat x = b (b: normal-equation rhs in hi precision) for n columns.
// x (hi) receives the solution.  final_check recomputes the residual in hi.
dl_status run_cg(dl_ctx* c, const Batch& B, const dl_solve_params& prm, Field* b, Field* x, bool final_check,
                 dl_solve_stats* stats, double* resid_out, bool x_init) {
  const int hi = prm.prec_hi, lo = prm.prec_lo, f = prm.flavour;
  const int n = ncols_of(B);
  dl_status s;
  if ((s = ensure_partial(c, B)) != DL_OK) return s;
  CGFields F;
  const int lo_ = lo;
  if ((s = ensure_field(c, "cg_r", lo_, B, &F.r)) || (s = ensure_field(c, "cg_p", lo_, B, &F.p)) ||
      (s = ensure_field(c, "cg_y", lo_, B, &F.y)) || (s = ensure_field(c, "cg_t1", lo_, B, &F.t1)) ||
      (s = ensure_field(c, "cg_q", lo_, B, &F.q)) || (s = ensure_field(c, "cg_t2", lo_, B, &F.t2)) ||
      (s = ensure_field(c, "cg_rh", hi, B, &F.rh)) || (s = ensure_field(c, "cg_ax", hi, B, &F.ax)) ||
      (s = ensure_field(c, "cg_th1", hi, B, &F.th1)) || (s = ensure_field(c, "cg_tq", hi, B, &F.tq)) ||
      (s = ensure_field(c, "cg_th2", hi, B, &F.th2)))
    return s;
  // |b|^2; x = 0 (r = b), or the caller's initial guess x (r = b - A x in the high precision)
  CK(dl::norm2(B, hi, b->ref(), nullptr, c->partial, c->st));
  CK(colsum(c, B, DL_S_RR0));
  if (x_init) {
    CK(normal_op(c, B, hi, f, x->ref(), F.th1->ref(), F.tq->ref(), F.th2->ref(), F.ax->ref(), nullptr));
    CK(dl::xmy_norm(B, hi, F.rh->ref(), b->ref(), F.ax->ref(), nullptr, c->partial, c->st));
    CK(colsum(c, B, DL_S_TMP));
  } else {
    CK(dl::zero(B, hi, x->ref(), nullptr, c->st));
  }
  CGState h;
  if ((s = download_state(c, n, h)) != DL_OK) return s;
  const double tol2_ = prm.tol * prm.tol;
  std::vector<int> nonfinite(n, 0);  // NaN or Inf in |b|^2 or the initial residual: not iterated
  for (int i = 0; i < n; ++i) {
    const double rr0 = h.S[DL_S_RR0 * DL_NCMAX + i];
    const double rr = x_init ? h.S[DL_S_TMP * DL_NCMAX + i] : rr0;
    h.S[DL_S_RR * DL_NCMAX + i] = rr;
    h.S[DL_S_MAXR * DL_NCMAX + i] = sqrt(rr);
    h.active[i] = (rr0 > 0.0 && rr > tol2_ * rr0) ? 1 : 0;
    h.flags[i] = 0;
    if (!std::isfinite(rr0) || !std::isfinite(rr)) {
      h.active[i] = 0;
      nonfinite[i] = 1;
    }
  }
  h.iters.assign(n, 0);
  CK(cudaMemcpyAsync(c->iters, h.iters.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemsetAsync(c->waitc, 0, DL_NCMAX * sizeof(int), c->st));
  if ((s = upload_state(c, n, h)) != DL_OK) return s;
  CK(dl::copy(B, lo, hi, F.r->ref(), x_init ? F.rh->ref() : b->ref(), nullptr, c->st));
  CK(dl::copy(B, lo, lo, F.p->ref(), F.r->ref(), nullptr, c->st));
  CK(dl::zero(B, lo, F.y->ref(), nullptr, c->st));
  const double tol2 = prm.tol * prm.tol;
  GraphEntry* ge = nullptr;
  if (c->use_graphs && (s = get_graph(c, B, lo, f, F, tol2, prm.delta, &ge)) != DL_OK) return s;
  const cudaGraphExec_t gexec = ge ? ge->exec : nullptr;
  const long long body_kernels = ge ? ge->kernels : 0;
  std::vector<int> finalized(n, 0), notconv(n, 0);
  for (int i = 0; i < n; ++i)
    if (!h.active[i]) finalized[i] = 1;  // zero right-hand side (x = 0) or an initial guess within tolerance
  int n_rel = 0;
  auto t0 = std::chrono::steady_clock::now();
  bool breakdown = false;
  for (int i = 0; i < n; ++i)
    if (nonfinite[i]) {
      breakdown = true;
      c->err = "non-finite source or initial residual in column " + std::to_string(i);
    }
  // a breakdown in low-precision arithmetic restarts the column from its true residual
  // (p = r after a reliable update), at most 8 times, when reliable updates are enabled
  std::vector<int> restarts(n, 0);
  while (true) {
    bool any = false;
    for (int i = 0; i < n; ++i) any |= (h.active[i] != 0);
    if (!any) break;
    int itmin = prm.max_iter;
    for (int i = 0; i < n; ++i)
      if (h.active[i]) itmin = std::min(itmin, h.iters[i]);
    const int ctr[2] = {0, std::max(1, std::min(prm.max_iter - itmin, 1 << 20))};
    CK(cudaMemcpyAsync(c->loopctr, ctr, sizeof(ctr), cudaMemcpyHostToDevice, c->st));
    int ran = 0;
    if (gexec) {
      CK(cudaGraphLaunch(gexec, c->st));
      CK(cudaMemcpyAsync(&ran, c->loopctr, sizeof(int), cudaMemcpyDeviceToHost, c->st));
      if ((s = download_state(c, n, h)) != DL_OK) return s;
      g_launches.fetch_add(body_kernels * ran);
      dl::stencil_tally_add(ge->tally, ran);
    } else {
      // the same body and loop condition launched from the host (profilers cannot
      // see kernel nodes inside conditional graphs); one readback per iteration
      int go = 1;
      while (go) {
        CK(cg_iteration(c, B, lo, f, F, tol2, prm.delta));
        CK(dl::cg_cond(n, c->active, c->flags, c->loopctr, c->loopctr + 1, c->waitc, 0, c->loopctr + 2, c->st));
        int hc[3];
        CK(cudaMemcpyAsync(hc, c->loopctr, sizeof(hc), cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        ran = hc[0];
        go = hc[2];
      }
      if ((s = download_state(c, n, h)) != DL_OK) return s;
    }
    std::vector<int> mask(n, 0);
    bool need = false;
    for (int i = 0; i < n; ++i) {
      if (finalized[i]) continue;
      if (h.flags[i] & DL_FLAG_BREAKDOWN) {
        char msg[256];
        snprintf(msg, sizeof(msg), "CG breakdown in column %d after %d iterations (pAp %.3e, rr %.3e, rr_new %.3e)", i,
                 h.iters[i], h.S[DL_S_PAP * DL_NCMAX + i], h.S[DL_S_RR * DL_NCMAX + i], h.S[DL_S_RRNEW * DL_NCMAX + i]);
        c->err = msg;
        mask[i] = 1;
        need = true;
        continue;
      }
      bool conv = (h.flags[i] & DL_FLAG_CONVERGED) != 0;
      bool upd = (h.flags[i] & DL_FLAG_UPDATE) != 0 && prm.delta > 0.0;
      bool maxed = h.active[i] && h.iters[i] >= prm.max_iter;
      if (maxed) {
        h.active[i] = 0;
        notconv[i] = 1;
      }
      if (conv || maxed || (upd && h.active[i])) {
        mask[i] = 1;
        need = true;
      }
    }
    if (getenv("DL_TRACE")) {
      for (int i = 0; i < n; ++i)
        fprintf(stderr, "[dl cg] col %d it %d active %d flags %d rr/rr0 %.3e pAp %.3e alpha %.3e beta %.3e maxr %.3e\n", i,
                h.iters[i], h.active[i], h.flags[i],
                h.S[DL_S_RR * DL_NCMAX + i] / std::max(h.S[DL_S_RR0 * DL_NCMAX + i], 1e-300),
                h.S[DL_S_PAP * DL_NCMAX + i], h.S[DL_S_ALPHA * DL_NCMAX + i], h.S[DL_S_BETA * DL_NCMAX + i],
                h.S[DL_S_MAXR * DL_NCMAX + i]);
    }
    if (!need) continue;
    std::vector<double> rr;
    if (prm.delta <= 0.0 && !final_check) {
      // no reliable updates and no final check (the TSM's truncated LP solves): a column that
      // stops only needs x += y; its true residual would decide nothing, so the normal
      // operator is not applied and the iterated residual stands for it
      CK(cudaMemcpyAsync(c->upd, mask.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c->st));
      CK(dl::accum(B, hi, lo, x->ref(), F.y->ref(), c->upd, 1, c->st));
      rr.assign(n, 0.0);
      for (int i = 0; i < n; ++i) rr[i] = h.S[DL_S_RR * DL_NCMAX + i];
    } else if ((s = reliable_update(c, B, hi, lo, f, F, x, b, mask, rr)) != DL_OK) {
      return s;
    }
    CK(cudaMemsetAsync(c->waitc, 0, DL_NCMAX * sizeof(int), c->st));
    // 16-bit search directions lose conjugacy over several decades: every reliable
    // update restarts them from the true residual (p = r).  FP32 ones are kept while the
    // true residual agrees with the iterated one; a column that went on iterating while
    // waiting for a batched update can take its iterated residual below the FP32 floor,
    // and a search direction kept across a true residual more than twice as large as the
    // iterated one (in norm) is no longer conjugate: it restarts too.
    if (lo == P16) {
      CK(dl::copy(B, lo, lo, F.p->ref(), F.r->ref(), c->upd, c->st));
    } else if (prm.delta > 0.0) {
      std::vector<int> dmask(n, 0);
      bool any_drift = false;
      for (int i = 0; i < n; ++i)
        if (mask[i] && !(h.flags[i] & DL_FLAG_BREAKDOWN) && rr[i] > 4.0 * h.S[DL_S_RR * DL_NCMAX + i]) {
          dmask[i] = 1;
          any_drift = true;
        }
      if (any_drift) {
        CK(cudaMemcpyAsync(c->upd, dmask.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c->st));
        CK(dl::copy(B, lo, lo, F.p->ref(), F.r->ref(), c->upd, c->st));
      }
    }
    {
      std::vector<int> rmask(n, 0);
      bool any_restart = false;
      for (int i = 0; i < n; ++i) {
        if (!mask[i] || !(h.flags[i] & DL_FLAG_BREAKDOWN)) continue;
        const double rr0 = h.S[DL_S_RR0 * DL_NCMAX + i];
        if (prm.delta > 0.0 && restarts[i] < 8 && rr[i] > prm.tol * prm.tol * rr0 && h.iters[i] < prm.max_iter &&
            std::isfinite(rr[i])) {
          ++restarts[i];
          h.flags[i] &= ~DL_FLAG_BREAKDOWN;
          h.active[i] = 1;
          rmask[i] = 1;
          any_restart = true;
        } else {
          breakdown = true;
        }
      }
      if (any_restart) {  // p = r (the true residual just copied to the Krylov precision)
        CK(cudaMemcpyAsync(c->upd, rmask.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c->st));
        CK(dl::copy(B, lo, lo, F.p->ref(), F.r->ref(), c->upd, c->st));
      }
    }
    for (int i = 0; i < n; ++i) {
      if (!mask[i]) continue;
      ++n_rel;
      double rr0 = h.S[DL_S_RR0 * DL_NCMAX + i];
      bool conv = (h.flags[i] & DL_FLAG_CONVERGED) != 0;
      h.flags[i] &= ~DL_FLAG_UPDATE;
      h.S[DL_S_RR * DL_NCMAX + i] = rr[i];
      h.S[DL_S_MAXR * DL_NCMAX + i] = sqrt(rr[i]);
      if (h.flags[i] & DL_FLAG_BREAKDOWN) {
        finalized[i] = 1;
        h.active[i] = 0;
      } else if (conv) {
        if (prm.delta > 0.0 && rr[i] > prm.tol * prm.tol * rr0 && h.iters[i] < prm.max_iter) {
          h.flags[i] &= ~DL_FLAG_CONVERGED;  // drifted: continue from the true residual
          h.active[i] = 1;
        } else {
          finalized[i] = 1;
        }
      } else if (notconv[i]) {
        finalized[i] = 1;
      }
    }
    if ((s = upload_state(c, n, h)) != DL_OK) return s;
  }
  // any column that never went through a final update
  {
    std::vector<int> mask(n, 0);
    bool need = false;
    for (int i = 0; i < n; ++i)
      if (!finalized[i]) {
        mask[i] = 1;
        need = true;
      }
    if (need) {
      CK(cudaMemcpyAsync(c->upd, mask.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c->st));
      CK(dl::accum(B, hi, lo, x->ref(), F.y->ref(), c->upd, 1, c->st));
    }
  }
  std::vector<double> resid(n, 0.0);
  if (final_check) {
    std::vector<int> all(n, 1);
    std::vector<double> rr;
    // y is zero here, so the update only recomputes the residual
    if ((s = reliable_update(c, B, hi, lo, f, F, x, b, all, rr)) != DL_OK) return s;
    for (int i = 0; i < n; ++i) {
      double rr0 = h.S[DL_S_RR0 * DL_NCMAX + i];
      resid[i] = rr0 > 0 ? sqrt(rr[i] / rr0) : 0.0;
    }
  } else {
    for (int i = 0; i < n; ++i) {
      double rr0 = h.S[DL_S_RR0 * DL_NCMAX + i];
      resid[i] = rr0 > 0 ? sqrt(h.S[DL_S_RR * DL_NCMAX + i] / rr0) : 0.0;
    }
  }
  CK(cudaStreamSynchronize(c->st));
  double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  const int plo = lo == PDF ? P64 : lo;  // profile slots: 0 high precision, 1 FP32, 2 16-bit
  if (c->profiling && plo <= P16 && c->prof_pending[plo]) {
    c->prof_pending[plo] = 0;
    if ((s = sample_stencil(c, B, lo, f, F)) != DL_OK) return s;
  }
  int maxit = 0;
  bool anync = false;
  for (int i = 0; i < n; ++i) {
    maxit = std::max(maxit, h.iters[i]);
    anync |= notconv[i] != 0;
  }
  if (stats) {
    for (int i = 0; i < n && i < DL_MAX_RHS; ++i) {
      stats->iters[i] = h.iters[i];
      stats->resid[i] = resid[i];
    }
    stats->reliable_updates = n_rel;
    stats->max_iters = maxit;
    stats->seconds = secs;
  }
  for (int i = 0; i < n; ++i)
    if (nonfinite[i]) resid[i] = std::numeric_limits<double>::quiet_NaN();
  if (stats)
    for (int i = 0; i < n && i < DL_MAX_RHS; ++i) stats->resid[i] = resid[i];
  if (resid_out)
    for (int i = 0; i < n; ++i) resid_out[i] = resid[i];
  c->last_iters.assign(h.iters.begin(), h.iters.begin() + n);
  c->last_resid = resid;
  if (breakdown) return DL_BREAKDOWN;
  if (anync) return fail(c, DL_NOT_CONVERGED, "max_iter reached");
  return DL_OK;
}

dl_status check_ctx(dl_ctx* c, bool need_gauge) {
  if (!c) return DL_ERR_ARG;
  if (c->lats.size() != 1) return fail(c, DL_ERR_STATE, "this call works on single-lattice contexts; use dl_batch_loops");
  if (need_gauge && !c->has_gauge) return fail(c, DL_ERR_STATE, "no gauge field loaded");
  return DL_OK;
}

int dtype_prec(int dtype) { return dtype == DL_C128 ? P64 : P32; }

// ---- solve pipeline on internal fields --------------------------------------
// From a full-lattice source (b_e, b_o, precision hi) to the solution
// (x_e, psi_o, precision hi).
dl_status solve_internal(dl_ctx* c, const Batch& B, const dl_solve_params& prm, Field* b_e, Field* b_o, Field* x_e,
                         Field* psi_o, bool final_check, dl_solve_stats* stats, bool x_init = false) {
  const int hi = prm.prec_hi, f = prm.flavour;
  dl_status s;
  Field *tmp_o, *bhat, *bn, *t2;
  if ((s = ensure_field(c, "sv_tmp_o", hi, B, &tmp_o)) || (s = ensure_field(c, "sv_bhat", hi, B, &bhat)) ||
      (s = ensure_field(c, "sv_bn", hi, B, &bn)) || (s = ensure_field(c, "sv_t2", hi, B, &t2)))
    return s;
  // bhat_e = b_e + kappa D_eo R_oo^{-1} b_o
  EpiSet Ei = epiB(B, CK_ONE, 2, f, 0, 0);
  CK(dl::twist(B, hi, tmp_o->ref(), b_o->ref(), Ei, nullptr, c->st));
  GaugeSet g{c->g64, c->g32, c->g16, c->gdf};
  EpiSet Ep = epiB(B, CK_K, 0, 0, 0, 0);
  CK(dl::dslash(B, hi, grec_of(c, hi), EPI_AUX, false, 0, tmp_o->ref(), b_e->ref(), bhat->ref(), g, Ep, nullptr, nullptr,
                NOF, NOF, NOF, nullptr, c->st));
  // bn = Mhat^dag bhat
  CK(stage1(c, B, hi, true, f, bhat->ref(), t2->ref(), nullptr));
  CK(stage2(c, B, hi, true, f, t2->ref(), bhat->ref(), bn->ref(), nullptr, nullptr));
  dl_status rs = run_cg(c, B, prm, bn, x_e, final_check, stats, nullptr, x_init);
  if (rs < 0) return rs;
  // psi_o = R_oo^{-1} (b_o + kappa D_oe x_e)
  EpiSet Er = epiB(B, CK_K, 2, f, 0, 0);
  CK(dl::dslash(B, hi, grec_of(c, hi), EPI_AUX, false, 1, x_e->ref(), b_o->ref(), psi_o->ref(), g, Er, nullptr, nullptr,
                NOF, NOF, NOF, nullptr, c->st));
  return rs;
}

// momentum list on the device for p2max
dl_status ensure_momenta(dl_ctx* c, int p2max) {
  if (c->mom_p2 == p2max) return DL_OK;
  int cnt = 0;
  dl_momenta(p2max, &cnt, nullptr);
  std::vector<int> lst(3 * cnt);
  dl_momenta(p2max, &cnt, lst.data());
  if (c->mom) cudaFree(c->mom);
  c->mom = nullptr;
  CK(cudaMalloc((void**)&c->mom, sizeof(int) * 3 * std::max(cnt, 1)));
  CK(cudaMemcpy(c->mom, lst.data(), sizeof(int) * 3 * cnt, cudaMemcpyHostToDevice));
  c->mom_p2 = p2max;
  c->np = cnt;
  return DL_OK;
}

int mom_extent(int p2max) {
  int m = 0;
  while ((m + 1) * (m + 1) <= p2max) ++m;
  return m;
}

// Contract (s_e, s_o) with (eta_e, eta_o) for estimator mode into out
// [ncol][T][np][nd][16] (device complex128) with the prefactor applied.
// B must describe one lattice segment (B.nlat == 1); its fields are read at the
// segment's offsets.
dl_status contract_internal(dl_ctx* c, const Batch& B, int prec, int mode, int with_deriv, int p2max, Field* s_e,
                            Field* s_o, Field* eta_e, Field* eta_o, double pre_re, double pre_im, double2* out,
                            int accumulate, Slices S = Slices{0, 1, 0}) {
  const LatDesc& L = B.lat[0];
  if (S.ns == 0) S = all_slices(L.T);
  dl_status s;
  if ((s = ensure_momenta(c, p2max)) != DL_OK) return s;
  const int m = mom_extent(p2max);
  const int mx = m, my = m, mz = m;  // the cube must hold every listed momentum
  const int NX = 2 * mx + 1, NY = 2 * my + 1, NZ = 2 * mz + 1;
  const int npad = 1 << L.lognpad;
  const int ncomp = with_deriv ? 80 : 16;
  const size_t V = 2ull * L.Vh;
  const bool fused = L.X <= 256;  // one CTA per (row, column group) holds X * cw <= 256 sites
  const size_t nW = fused ? 0 : (size_t)ncomp * V * npad;
  const size_t nG1 = (size_t)ncomp * S.ns * L.Z * L.Y * NX * npad;
  const size_t nG2 = (size_t)ncomp * S.ns * L.Z * NY * NX * npad;
  const size_t nG3 = (size_t)ncomp * S.ns * NZ * NY * NX * npad;
  const size_t nph = 17 * 256 + 64;  // phase tables (x: up to 17 momenta x 256 sites of 16-byte pairs)
  if ((s = ensure_scratch(c, sizeof(double2) * (nW + nG1 + nG2 + nG3 + nph))) != DL_OK) return s;
  double2* W = (double2*)c->scratch;
  double2* G1 = W + nW;
  double2* G2 = G1 + nG1;
  double2* G3 = G2 + nG2;
  double2* ph = G3 + nG3;
  if (L.X > (int)nph || L.Y > (int)nph || L.Z > (int)nph) return fail(c, DL_ERR_ARG, "spatial extent too large");
  // arithmetic of the DFT buffers: 1 float, 2 double-float, 0 double (the unfused fallback)
  const int fp32 = !fused ? 0 : (prec == P32 ? 1 : (prec == PDF ? 2 : 0));
  if (fused) {
    CK(dl::contract_x(B, prec, mode, with_deriv, s_e->ref(), s_o->ref(), eta_e ? eta_e->ref() : NOF,
                      eta_o ? eta_o->ref() : NOF, prec == PDF ? c->gdf : c->g64, c->g32, c->rec32, mx, ph, G1, S,
                      c->st));
  } else {
    if (S.ns != L.T) return fail(c, DL_ERR_ARG, "slice-restricted contractions need X <= 256");
    CK(dl::contract_sites(B, prec, mode, with_deriv, s_e->ref(), s_o->ref(), eta_e ? eta_e->ref() : NOF,
                          eta_o ? eta_o->ref() : NOF, c->g64, W, c->st));
    CK(dl::dft_pass(W, G1, (long long)ncomp * L.T * L.Z * L.Y, L.X, npad, mx, ph, fp32, c->st));
  }
  CK(dl::dft_pass(G1, G2, (long long)ncomp * S.ns * L.Z, L.Y, (long long)NX * npad, my, ph, fp32, c->st));
  CK(dl::dft_pass(G2, G3, (long long)ncomp * S.ns, L.Z, (long long)NY * NX * npad, mz, ph, fp32, c->st));
  CK(dl::contract_finalize(B, with_deriv, c->np, c->mom, mx, my, mz, G3, fp32, pre_re, pre_im, out, accumulate, S,
                           c->st));
  return DL_OK;
}

// w = (BH)^k s on the full lattice, B = R_f^{-1}, H = -kappa D (Eq. HPE)
dl_status bh_power(dl_ctx* c, const Batch& B, int prec, int f, int k, Field* se, Field* so, Field** we, Field** wo) {
  dl_status s;
  Field *ae, *ao, *be, *bo;
  if ((s = ensure_field(c, "bh_ae", prec, B, &ae)) || (s = ensure_field(c, "bh_ao", prec, B, &ao)) ||
      (s = ensure_field(c, "bh_be", prec, B, &be)) || (s = ensure_field(c, "bh_bo", prec, B, &bo)))
    return s;
  GaugeSet g{c->g64, c->g32, c->g16, c->gdf};
  EpiSet E = epiB(B, CK_MK, 2, f, 0, 0);
  Field *ie = se, *io = so;
  for (int it = 0; it < k; ++it) {
    Field* oe = (it % 2 == 0) ? ae : be;
    Field* oo = (it % 2 == 0) ? ao : bo;
    CK(dl::dslash(B, prec, grec_of(c, prec), EPI_PLAIN, false, 0, io->ref(), NOF, oe->ref(), g, E, nullptr, nullptr, NOF,
                  NOF, NOF, nullptr, c->st));
    CK(dl::dslash(B, prec, grec_of(c, prec), EPI_PLAIN, false, 1, ie->ref(), NOF, oo->ref(), g, E, nullptr, nullptr, NOF,
                  NOF, NOF, nullptr, c->st));
    ie = oe;
    io = oo;
  }
  *we = ie;
  *wo = io;
  return DL_OK;
}

}  // namespace dlh

using namespace dlh;

// ============================================================================
extern "C" {

static dl_status create_ctx(dl_ctx** out, int nlat, const int* dims, int device, void* cuda_stream) {
  if (!out || !dims || nlat < 1 || nlat > DL_MAX_LAT) return DL_ERR_ARG;
  *out = nullptr;
  long long Vt = 0;
  for (int l = 0; l < nlat; ++l) {
    for (int k = 0; k < 4; ++k)
      if (dims[4 * l + k] < 2 || (dims[4 * l + k] & 1)) return DL_ERR_ARG;
    Vt += (long long)dims[4 * l] * dims[4 * l + 1] * dims[4 * l + 2] * dims[4 * l + 3] / 2;
  }
  if (Vt >= (1LL << 31) / DL_MAXC) return DL_ERR_ARG;
  dl_ctx* c = new dl_ctx();
  c->dev = device;
  long long off = 0;
  for (int l = 0; l < nlat; ++l) {
    LatInfo L;
    memcpy(L.dims, dims + 4 * l, sizeof(int) * 4);
    L.Vh = (int)((long long)L.dims[0] * L.dims[1] * L.dims[2] * L.dims[3] / 2);
    L.gsite_off = off;
    off += L.Vh;
    c->lats.push_back(L);
  }
  c->Vh_total = Vt;
  memcpy(c->dims, dims, sizeof(int) * 4);
  c->Vh = c->lats[0].Vh;
  // blocks of any launch: 256-thread blocks over <= 32 columns of every site, one
  // ragged block per lattice segment
  c->partial_blocks = ((size_t)Vt * DL_MAXC + 255) / 256 + 2 * DL_MAX_LAT + 8;
  c->user = (cudaStream_t)cuda_stream;
  {
    const char* gv = getenv("DL_GRAPHS");  // "0": launch the CG loop from the host (for profilers)
    c->use_graphs = !(gv && gv[0] == '0');
  }
  cudaError_t e;
  if ((e = cudaSetDevice(device)) != cudaSuccess || (e = cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaMalloc((void**)&c->S, sizeof(double) * DL_NS * DL_NCMAX)) != cudaSuccess ||
      (e = cudaMalloc((void**)&c->active, sizeof(int) * DL_NCMAX)) != cudaSuccess ||
      (e = cudaMalloc((void**)&c->flags, sizeof(int) * DL_NCMAX)) != cudaSuccess ||
      (e = cudaMalloc((void**)&c->iters, sizeof(int) * DL_NCMAX)) != cudaSuccess ||
      (e = cudaMalloc((void**)&c->upd, sizeof(int) * DL_NCMAX)) != cudaSuccess ||
      (e = cudaMalloc((void**)&c->misc, sizeof(double2) * 4096)) != cudaSuccess ||
      (e = cudaMalloc((void**)&c->partial, sizeof(double) * DL_MAXC * c->partial_blocks)) != cudaSuccess ||
      (e = cudaMalloc((void**)&c->loopctr, 3 * sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc((void**)&c->waitc, DL_NCMAX * sizeof(int))) != cudaSuccess) {
    dl_destroy(c);
    return e == cudaErrorMemoryAllocation ? DL_ERR_OOM : DL_ERR_CUDA;
  }
  for (int k = 0; k < 8; ++k)
    if ((e = cudaEventCreate(&c->pev[k])) != cudaSuccess) {
      dl_destroy(c);
      return DL_ERR_CUDA;
    }
  *out = c;
  return DL_OK;
}

dl_status dl_create(dl_ctx** out, const int dims[4], int device, void* cuda_stream) try {
  return create_ctx(out, 1, dims, device, cuda_stream);
} DL_CATCH(nullptr)

dl_status dl_create_multi(dl_ctx** out, int nlat, const int* dims, int device, void* cuda_stream) try {
  return create_ctx(out, nlat, dims, device, cuda_stream);
} DL_CATCH(nullptr)

void dl_destroy(dl_ctx* c) try {
  if (!c) return;
  cudaSetDevice(c->dev);
  if (c->st) cudaStreamSynchronize(c->st);
  invalidate_graphs(c);
  for (auto& kv : c->ws) {
    cudaFree(kv.second.data);
    if (kv.second.norm) cudaFree(kv.second.norm);
  }
  for (auto& kv : c->bufs)
    if (kv.second.p) cudaFree(kv.second.p);
  void* ptrs[] = {c->waitc, c->loopctr, c->g64, c->gdf, c->g32, c->g16, c->partial, c->S, c->active, c->flags, c->iters, c->upd, c->misc, c->mom,
                  c->scratch};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (int k = 0; k < 8; ++k)
    if (c->pev[k]) cudaEventDestroy(c->pev[k]);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->st) cudaStreamDestroy(c->st);
  delete c;
} catch (...) {
}

const char* dl_last_error(const dl_ctx* c) { return c ? c->err.c_str() : "null context"; }

dl_status dl_set_stream(dl_ctx* c, void* s) try {
  if (!c) return DL_ERR_ARG;
  c->user = (cudaStream_t)s;
  return DL_OK;
} DL_CATCH(c)

dl_status dl_load_gauge_lat(dl_ctx* c, int lat, const double* links, int on_device, double t_boundary, int recon_f32,
                            int recon_f16) try {
  if (!c || !links || lat < 0 || lat >= (int)c->lats.size()) return DL_ERR_ARG;
  if (!(recon_f32 == 12 || recon_f32 == 8 || recon_f32 == 18)) return fail(c, DL_ERR_ARG, "recon_f32 must be 18, 12 or 8");
  if (!(recon_f16 == 12 || recon_f16 == 8)) return fail(c, DL_ERR_ARG, "recon_f16 must be 12 or 8");
  if (recon_f32 == 18) recon_f32 = 12;  // FP32 operator reads the 12-real form; 18 is accepted as "uncompressed request"
  bool any = false;
  for (auto& L : c->lats) any |= L.has_gauge;
  if (any && (recon_f32 != c->rec32 || recon_f16 != c->rec16))
    return fail(c, DL_ERR_ARG, "every lattice of a context uses the same link compression");
  dl_status s;
  if ((s = enter(c)) != DL_OK) return s;
  const size_t nl_total = 2ull * c->Vh_total * 4;
  if (!c->g64) {
    CK(cudaMalloc(&c->g64, nl_total * 9 * sizeof(double2)));  // 144 B per link
    CK(cudaMalloc(&c->gdf, nl_total * 9 * sizeof(float4)));   // 144 B per link
    CK(cudaMalloc(&c->g32, nl_total * 3 * sizeof(float4)));    // up to 48 B per link
    CK(cudaMalloc(&c->g16, nl_total * 3 * sizeof(uint2)));     // up to 24 B per link
  }
  LatInfo& LI = c->lats[lat];
  const size_t nl = 2ull * LI.Vh * 4;
  const double* dlinks = links;
  void* tmp = nullptr;
  if (!on_device) {
    CK(cudaMalloc(&tmp, nl * 9 * sizeof(double2)));
    CK(cudaMemcpyAsync(tmp, links, nl * 9 * sizeof(double2), cudaMemcpyHostToDevice, c->st));
    dlinks = (const double*)tmp;
  }
  LI.tbc = t_boundary;
  c->rec32 = recon_f32;
  c->rec16 = recon_f16;
  LatDesc L;
  memset(&L, 0, sizeof(L));
  L.X = LI.dims[0];
  L.Y = LI.dims[1];
  L.Z = LI.dims[2];
  L.T = LI.dims[3];
  L.Vh = LI.Vh;
  // byte offsets of this lattice in each gauge array (chunk bytes x chunks per link x 8 links per parity site)
  const size_t o = (size_t)LI.gsite_off;
  char* g64 = (char*)c->g64 + o * 16 * 9 * 8;
  char* gdf = (char*)c->gdf + o * 16 * 9 * 8;
  char* g32 = (char*)c->g32 + o * 16 * (recon_f32 == 12 ? 3 : 2) * 8;
  char* g16 = (char*)c->g16 + o * (recon_f16 == 12 ? 8 * 3 : 16 * 1) * 8;
  cudaError_t e = dl::pack_gauge(L, dlinks, g64, gdf, g32, recon_f32, g16, recon_f16, c->st);
  if (tmp) {
    cudaStreamSynchronize(c->st);
    cudaFree(tmp);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "pack_gauge");
  LI.has_gauge = true;
  if (lat == 0) c->tbc = t_boundary;
  c->has_gauge = true;
  for (auto& Lx : c->lats) c->has_gauge = c->has_gauge && Lx.has_gauge;
  invalidate_graphs(c);
  return leave(c);
} DL_CATCH(c)

dl_status dl_load_gauge(dl_ctx* c, const double* links, int on_device, double t_boundary, int recon_f32, int recon_f16) try {
  return dl_load_gauge_lat(c, 0, links, on_device, t_boundary, recon_f32, recon_f16);
} DL_CATCH(c)

dl_status dl_set_params_lat(dl_ctx* c, int lat, double kappa, double amu) try {
  if (!c || lat < 0 || lat >= (int)c->lats.size()) return DL_ERR_ARG;
  if (!(kappa > 0.0) || !std::isfinite(kappa) || !std::isfinite(amu)) return fail(c, DL_ERR_ARG, "bad kappa/amu");
  c->lats[lat].kappa = kappa;
  c->lats[lat].amu = amu;
  if (lat == 0) {
    c->kappa = kappa;
    c->amu = amu;
  }
  return DL_OK;
} DL_CATCH(c)

dl_status dl_set_params(dl_ctx* c, double kappa, double amu) try {
  if (!c) return DL_ERR_ARG;
  for (int l = 0; l < (int)c->lats.size(); ++l) {
    dl_status s = dl_set_params_lat(c, l, kappa, amu);
    if (s != DL_OK) return s;
  }
  return DL_OK;
} DL_CATCH(c)

dl_status dl_noise_z4(dl_ctx* c, uint64_t seed, uint64_t first_index, int n, void* out, int dtype, int quadrant) try {
  if (!c || !out || n < 1 || n > DL_MAX_RHS || (dtype != DL_C128 && dtype != DL_C64)) return DL_ERR_ARG;
  dl_status s;
  if ((s = check_ctx(c, false)) != DL_OK) return s;
  if ((s = enter(c)) != DL_OK) return s;
  const int prec = dtype_prec(dtype);
  Batch B = make_batch(c, n);
  Field *e, *o;
  if ((s = ensure_field(c, "nz_e", prec, B, &e)) || (s = ensure_field(c, "nz_o", prec, B, &o))) return s;
  CK(dl::noise_z4(B, prec, 0, e->ref(), seed, first_index, quadrant, c->st));
  CK(dl::noise_z4(B, prec, 1, o->ref(), seed, first_index, quadrant, c->st));
  CK(dl::unpack(B, prec, 0, out, e->ref(), dtype, c->st));
  CK(dl::unpack(B, prec, 1, out, o->ref(), dtype, c->st));
  return leave(c);
} DL_CATCH(c)

// Time dilution (Sec. 2.3): the noise of dl_noise_z4 on the slices t = t0 (mod dt), zero
// elsewhere.  The natural layout [n][T][Z][Y][X][4][3] keeps each time slice of each column
// contiguous, so the cleared slices are byte ranges of `out`: consecutive ones (also across
// columns) are merged and cleared by one memset each.
dl_status dl_noise_z4_tdil(dl_ctx* c, uint64_t seed, uint64_t first_index, int n, void* out, int dtype, int quadrant,
                           int t0, int dt) try {
  dl_status s;
  if ((s = check_ctx(c, false)) != DL_OK) return s;
  const int T = c->dims[3];
  if (dt < 1 || dt > T || t0 < 0 || t0 >= dt)
    return fail(c, DL_ERR_ARG, "dl_noise_z4_tdil: need 1 <= dt <= T and 0 <= t0 < dt");
  if ((s = dl_noise_z4(c, seed, first_index, n, out, dtype, quadrant)) != DL_OK) return s;
  if ((s = enter(c)) != DL_OK) return s;
  const size_t slice = (size_t)c->dims[0] * c->dims[1] * c->dims[2] * 12 * (dtype == DL_C128 ? 16 : 8);
  char* base = static_cast<char*>(out);
  const long long nslices = (long long)n * T;  // out holds exactly n * T slices
  long long run = -1;                           // first slice of the run being cleared
  for (long long j = 0; j <= nslices; ++j) {
    const bool clear = j < nslices && (int)(j % T) % dt != t0;
    if (clear && run < 0) run = j;
    if (!clear && run >= 0) {
      CK(cudaMemsetAsync(base + (size_t)run * slice, 0, (size_t)(j - run) * slice, c->st));
      run = -1;
    }
  }
  return leave(c);
} DL_CATCH(c)

dl_status dl_apply(dl_ctx* c, int op, int prec, int f, int n, const void* in, const void* aux, void* out, int dtype) try {
  dl_status s;
  if ((s = check_ctx(c, true)) != DL_OK) return s;
  if (!in || !out || n < 1 || n > DL_MAX_RHS || (f != 1 && f != -1) || prec_rank(prec) < 0 ||
      (dtype != DL_C128 && dtype != DL_C64))
    return fail(c, DL_ERR_ARG, "dl_apply: bad argument");
  if (op == DL_OP_RECON && !aux) return fail(c, DL_ERR_ARG, "DL_OP_RECON needs aux");
  prec = internal_prec(prec);
  if ((s = enter(c)) != DL_OK) return s;
  Batch B = make_batch(c, n);
  if ((s = ensure_partial(c, B)) != DL_OK) return s;
  Field *ie, *io, *oe, *oo, *ae, *ao, *t;
  if ((s = ensure_field(c, "ap_ie", prec, B, &ie)) || (s = ensure_field(c, "ap_io", prec, B, &io)) ||
      (s = ensure_field(c, "ap_oe", prec, B, &oe)) || (s = ensure_field(c, "ap_oo", prec, B, &oo)) ||
      (s = ensure_field(c, "ap_ae", prec, B, &ae)) || (s = ensure_field(c, "ap_ao", prec, B, &ao)) ||
      (s = ensure_field(c, "ap_t", prec, B, &t)))
    return s;
  CK(dl::pack(B, prec, 0, ie->ref(), in, dtype, c->st));
  CK(dl::pack(B, prec, 1, io->ref(), in, dtype, c->st));
  if (aux) {
    CK(dl::pack(B, prec, 0, ae->ref(), aux, dtype, c->st));
    CK(dl::pack(B, prec, 1, ao->ref(), aux, dtype, c->st));
  }
  GaugeSet g{c->g64, c->g32, c->g16, c->gdf};
  const int gr = grec_of(c, prec);
  auto D = [&](int epi_kind, bool dag, int par, Field* src, Field* ax, Field* dst, const EpiSet& E) {
    return dl::dslash(B, prec, gr, epi_kind, dag, par, src->ref(), ax ? ax->ref() : NOF, dst->ref(), g, E, nullptr,
                      nullptr, NOF, NOF, NOF, nullptr, c->st);
  };
  switch (op) {
    case DL_OP_M:
    case DL_OP_MDAG: {
      bool dag = op == DL_OP_MDAG;
      EpiSet E = epiB(B, CK_MK, 0, 0, 1, dag ? -f : f);
      CK(D(EPI_AUX, dag, 0, io, ie, oe, E));
      CK(D(EPI_AUX, dag, 1, ie, io, oo, E));
      break;
    }
    case DL_OP_HOP: {
      EpiSet E = epiB(B, CK_ONE, 0, 0, 0, 0);
      CK(D(EPI_PLAIN, false, 0, io, nullptr, oe, E));
      CK(D(EPI_PLAIN, false, 1, ie, nullptr, oo, E));
      break;
    }
    case DL_OP_MHAT:
    case DL_OP_MHAT_DAG: {
      bool dag = op == DL_OP_MHAT_DAG;
      CK(stage1(c, B, prec, dag, f, ie->ref(), t->ref(), nullptr));
      CK(stage2(c, B, prec, dag, f, t->ref(), ie->ref(), oe->ref(), nullptr, nullptr));
      CK(dl::zero(B, prec, oo->ref(), nullptr, c->st));
      break;
    }
    case DL_OP_PREP: {
      EpiSet Ei = epiB(B, CK_ONE, 2, f, 0, 0);
      CK(dl::twist(B, prec, t->ref(), io->ref(), Ei, nullptr, c->st));
      EpiSet E = epiB(B, CK_K, 0, 0, 0, 0);
      CK(D(EPI_AUX, false, 0, t, ie, oe, E));
      CK(dl::zero(B, prec, oo->ref(), nullptr, c->st));
      break;
    }
    case DL_OP_RECON: {
      CK(dl::copy(B, prec, prec, oe->ref(), ie->ref(), nullptr, c->st));
      EpiSet E = epiB(B, CK_K, 2, f, 0, 0);
      CK(D(EPI_AUX, false, 1, ie, ao, oo, E));
      break;
    }
    case DL_OP_BH: {
      EpiSet E = epiB(B, CK_MK, 2, f, 0, 0);
      CK(D(EPI_PLAIN, false, 0, io, nullptr, oe, E));
      CK(D(EPI_PLAIN, false, 1, ie, nullptr, oo, E));
      break;
    }
    default:
      return fail(c, DL_ERR_ARG, "unknown operator");
  }
  CK(dl::unpack(B, prec, 0, out, oe->ref(), dtype, c->st));
  CK(dl::unpack(B, prec, 1, out, oo->ref(), dtype, c->st));
  return leave(c);
} DL_CATCH(c)

dl_status dl_solve(dl_ctx* c, const void* src, void* sol, int n, int dtype, const dl_solve_params* prm,
                   dl_solve_stats* stats) try {
  dl_status s;
  if ((s = check_ctx(c, true)) != DL_OK) return s;
  if (!src || !sol || !prm || n < 1 || n > DL_MAX_RHS || (dtype != DL_C128 && dtype != DL_C64))
    return fail(c, DL_ERR_ARG, "dl_solve: bad argument");
  if (prec_rank(prm->prec_hi) < 0 || prec_rank(prm->prec_hi) > 1 || prec_rank(prm->prec_lo) < prec_rank(prm->prec_hi) ||
      !(prm->tol > 0.0) || prm->max_iter < 1 || (prm->flavour != 1 && prm->flavour != -1) || prm->delta < 0.0 ||
      prm->delta >= 1.0)
    return fail(c, DL_ERR_ARG, "dl_solve: bad parameters");
  if ((s = enter(c)) != DL_OK) return s;
  dl_solve_params sp = *prm;
  sp.prec_hi = internal_prec(prm->prec_hi);
  sp.prec_lo = internal_prec(prm->prec_lo);
  prm = &sp;
  const int hi = prm->prec_hi;
  Batch B = make_batch(c, n);
  if ((s = ensure_partial(c, B)) != DL_OK) return s;
  Field *be, *bo, *xe, *po;
  if ((s = ensure_field(c, "sl_be", hi, B, &be)) || (s = ensure_field(c, "sl_bo", hi, B, &bo)) ||
      (s = ensure_field(c, "sl_xe", hi, B, &xe)) || (s = ensure_field(c, "sl_po", hi, B, &po)))
    return s;
  CK(dl::pack(B, hi, 0, be->ref(), src, dtype, c->st));
  CK(dl::pack(B, hi, 1, bo->ref(), src, dtype, c->st));
  dl_solve_stats st;
  memset(&st, 0, sizeof(st));
  dl_status rs = solve_internal(c, B, *prm, be, bo, xe, po, true, &st);
  if (rs < 0) return rs;
  CK(dl::unpack(B, hi, 0, sol, xe->ref(), dtype, c->st));
  CK(dl::unpack(B, hi, 1, sol, po->ref(), dtype, c->st));
  // true residual |b - M psi| / |b| on the full lattice, in the solve's high
  // precision with FP64 reductions
  {
    Field *bh_e, *bh_o, *re, *ro;
    if ((s = ensure_field(c, "tr_be", hi, B, &bh_e)) || (s = ensure_field(c, "tr_bo", hi, B, &bh_o)) ||
        (s = ensure_field(c, "tr_re", hi, B, &re)) || (s = ensure_field(c, "tr_ro", hi, B, &ro)))
      return s;
    CK(dl::pack(B, hi, 0, bh_e->ref(), src, dtype, c->st));
    CK(dl::pack(B, hi, 1, bh_o->ref(), src, dtype, c->st));
    GaugeSet g{c->g64, c->g32, c->g16, c->gdf};
    EpiSet E = epiB(B, CK_MK, 0, 0, 1, prm->flavour);
    CK(dl::dslash(B, hi, grec_of(c, hi), EPI_AUX, false, 0, po->ref(), xe->ref(), re->ref(), g, E, nullptr, nullptr, NOF,
                  NOF, NOF, nullptr, c->st));
    CK(dl::dslash(B, hi, grec_of(c, hi), EPI_AUX, false, 1, xe->ref(), po->ref(), ro->ref(), g, E, nullptr, nullptr, NOF,
                  NOF, NOF, nullptr, c->st));
    std::vector<double> S(DL_NS * DL_NCMAX);
    double num[DL_MAX_RHS] = {0}, den[DL_MAX_RHS] = {0};
    auto col_sum = [&](double* acc) -> dl_status {
      CK(colsum(c, B, DL_S_TMP));
      CK(cudaMemcpyAsync(S.data(), c->S, sizeof(double) * DL_NS * DL_NCMAX, cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
      for (int i = 0; i < n; ++i) acc[i] += S[DL_S_TMP * DL_NCMAX + i];
      return DL_OK;
    };
    CK(dl::xmy_norm(B, hi, re->ref(), bh_e->ref(), re->ref(), nullptr, c->partial, c->st));
    if ((s = col_sum(num)) != DL_OK) return s;
    CK(dl::xmy_norm(B, hi, ro->ref(), bh_o->ref(), ro->ref(), nullptr, c->partial, c->st));
    if ((s = col_sum(num)) != DL_OK) return s;
    CK(dl::norm2(B, hi, bh_e->ref(), nullptr, c->partial, c->st));
    if ((s = col_sum(den)) != DL_OK) return s;
    CK(dl::norm2(B, hi, bh_o->ref(), nullptr, c->partial, c->st));
    if ((s = col_sum(den)) != DL_OK) return s;
    for (int i = 0; i < n; ++i) st.true_resid[i] = den[i] > 0 ? sqrt(num[i] / den[i]) : 0.0;
  }
  if (stats) *stats = st;
  dl_status ls = leave(c);
  if (ls != DL_OK) return ls;
  return rs;
} DL_CATCH(c)

dl_status dl_profile(dl_ctx* c, int enable, double* out) try {
  if (!c) return DL_ERR_ARG;
  if (out) {
    for (int k = 0; k < 4; ++k)
      for (int p = 0; p < 3; ++p) {
        out[(k * 3 + p) * 3 + 0] = (double)c->prof_n[k][p];
        out[(k * 3 + p) * 3 + 1] = c->prof_ms[k][p];
        out[(k * 3 + p) * 3 + 2] = (double)c->prof_items[k][p];
      }
  }
  if (enable >= 0) {
    if ((enable != 0) != (c->profiling != 0)) invalidate_graphs(c);
    dl::stencil_prof_enable(enable != 0);
    c->profiling = enable != 0;
    c->prof_pending[0] = c->prof_pending[1] = c->prof_pending[2] = c->profiling;
    memset(c->prof_ms, 0, sizeof(c->prof_ms));
    memset(c->prof_n, 0, sizeof(c->prof_n));
    memset(c->prof_items, 0, sizeof(c->prof_items));
  }
  return DL_OK;
} DL_CATCH(c)

long long dl_kernel_launches(void) { return g_launches.load(); }

dl_status dl_profile_stencils(double* out) try {
  if (!out) return DL_ERR_ARG;
  return dl::stencil_prof_read(out) == cudaSuccess ? DL_OK : DL_ERR_CUDA;
} DL_CATCH(nullptr)

dl_status dl_momenta(int p2max, int* count, int* list) try {
  if (!count || p2max < 0 || p2max > 64) return DL_ERR_ARG;
  int m = mom_extent(p2max);
  int k = 0;
  for (int nz = -m; nz <= m; ++nz)
    for (int ny = -m; ny <= m; ++ny)
      for (int nx = -m; nx <= m; ++nx)
        if (nx * nx + ny * ny + nz * nz <= p2max) {
          if (list) {
            list[3 * k] = nx;
            list[3 * k + 1] = ny;
            list[3 * k + 2] = nz;
          }
          ++k;
        }
  *count = k;
  return DL_OK;
} DL_CATCH(nullptr)

// dl_contract and dl_contract_slices: pack the natural fields, apply (BH)^4 for the HPE
// estimator, contract on the slices S
static dl_status contract_api(dl_ctx* c, int est, const void* eta, const void* sol, int n, int dtype, int with_deriv,
                              int p2max, double* out, int accumulate, Slices S) {
  dl_status s;
  if ((s = check_ctx(c, true)) != DL_OK) return s;
  if (!sol || !out || n < 1 || n > DL_MAX_RHS || est < 0 || est > 3 || p2max < 0 || p2max > 64 ||
      (dtype != DL_C128 && dtype != DL_C64))
    return fail(c, DL_ERR_ARG, "dl_contract: bad argument");
  if ((est == DL_EST_STANDARD || est == DL_EST_GEN || est == DL_EST_HPE) && !eta)
    return fail(c, DL_ERR_ARG, "estimator needs eta");
  if (est == DL_EST_HPE && with_deriv) return fail(c, DL_ERR_ARG, "the HPE estimator is local only");
  if ((s = enter(c)) != DL_OK) return s;
  const int prec = dtype == DL_C128 ? PDF : P32;  // complex128 inputs are contracted in double-float
  Batch B = make_batch(c, n);
  Field *se, *so, *ee, *eo;
  if ((s = ensure_field(c, "ct_se", prec, B, &se)) || (s = ensure_field(c, "ct_so", prec, B, &so)) ||
      (s = ensure_field(c, "ct_ee", prec, B, &ee)) || (s = ensure_field(c, "ct_eo", prec, B, &eo)))
    return s;
  CK(dl::pack(B, prec, 0, se->ref(), sol, dtype, c->st));
  CK(dl::pack(B, prec, 1, so->ref(), sol, dtype, c->st));
  if (eta) {
    CK(dl::pack(B, prec, 0, ee->ref(), eta, dtype, c->st));
    CK(dl::pack(B, prec, 1, eo->ref(), eta, dtype, c->st));
  } else {
    CK(dl::zero(B, prec, ee->ref(), nullptr, c->st));
    CK(dl::zero(B, prec, eo->ref(), nullptr, c->st));
  }
  Field *we = se, *wo = so;
  if (est == DL_EST_HPE)
    if ((s = bh_power(c, B, prec, 1, 4, se, so, &we, &wo)) != DL_OK) return s;
  double pre_re = 1.0, pre_im = 0.0;
  if (est == DL_EST_ONE_END) {
    pre_re = 0.0;
    pre_im = -4.0 * c->kappa * c->amu;
  } else if (est == DL_EST_GEN) {
    pre_re = 2.0;
  }
  if ((s = contract_internal(c, B, prec, est, with_deriv, p2max, we, wo, ee, eo, pre_re, pre_im, (double2*)out,
                             accumulate, S)) != DL_OK)
    return s;
  return leave(c);
}

dl_status dl_contract(dl_ctx* c, int est, const void* eta, const void* sol, int n, int dtype, int with_deriv, int p2max,
                      double* out, int accumulate) try {
  if (!c) return DL_ERR_ARG;
  return contract_api(c, est, eta, sol, n, dtype, with_deriv, p2max, out, accumulate, all_slices(c->dims[3]));
} DL_CATCH(c)

dl_status dl_contract_slices(dl_ctx* c, int est, const void* eta, const void* sol, int n, int dtype, int p2max, int t0,
                             int dt, double* out, int accumulate) try {
  if (!c) return DL_ERR_ARG;
  const int T = c->dims[3];
  if (dt < 1 || dt > T || t0 < 0 || t0 >= dt)
    return fail(c, DL_ERR_ARG, "dl_contract_slices: need 1 <= dt <= T and 0 <= t0 < dt");
  return contract_api(c, est, eta, sol, n, dtype, 0, p2max, out, accumulate, Slices{t0, dt, (T - 1 - t0) / dt + 1});
} DL_CATCH(c)

// The closed form of the exact HPE orders counts only the back-and-forth paths of two
// hops; on a lattice with an extent of 2 two forward hops also return to the site
// (through two different links), so the form is exact only for extents >= 4.
static bool hpe_exact_valid(const dl_ctx* c) {
  for (const auto& L : c->lats)
    for (int k = 0; k < 4; ++k)
      if (L.dims[k] < 4) return false;
  return true;
}

dl_status dl_hpe_exact(dl_ctx* c, int flavour, double* out16) try {
  if (!c || !out16 || (flavour != 1 && flavour != -1)) return DL_ERR_ARG;
  if (!hpe_exact_valid(c))
    return fail(c, DL_ERR_ARG, "dl_hpe_exact: every lattice extent must be at least 4 (with an extent of 2, two "
                               "forward hops return to the site and the closed form misses those paths)");
  dl_status s;
  if ((s = enter(c)) != DL_OK) return s;
  CK(dl::hpe_exact(c->kappa, c->amu, flavour, c->misc, c->st));
  CK(cudaMemcpyAsync(out16, c->misc, sizeof(double2) * 16, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  return leave(c);
} DL_CATCH(c)

dl_status dl_tsm_run(dl_ctx* c, const dl_tsm_params* prm, double* loops, double* obs_hp, double* obs_lp_pair,
                     double* obs_lp, dl_tsm_info* info) try {
  dl_status s;
  if ((s = check_ctx(c, true)) != DL_OK) return s;
  if (!prm || prm->n_hp < 0 || prm->n_lp < 0 || prm->n_hp + prm->n_lp < 1 || prm->block < 0 || prm->block > DL_MAX_RHS ||
      !(prm->tol_hp > 0.0) || !(prm->tol_lp > 0.0) || prm->p2max < 0 || prm->p2max > 64 || prm->max_iter < 1 ||
      prm->prec_hp_lo < DL_F64 || prm->prec_hp_lo > DL_F16 || prm->prec_lp_lo < DL_F32 || prm->prec_lp_lo > DL_F16 ||
      prm->delta_hp < 0.0 || prm->delta_hp >= 1.0)
    return fail(c, DL_ERR_ARG, "dl_tsm_run: bad parameters");
  if (prm->hpe && prm->with_deriv) return fail(c, DL_ERR_ARG, "dl_tsm_run: the HPE estimator is local only");
  if (prm->hpe && !hpe_exact_valid(c))
    return fail(c, DL_ERR_ARG, "dl_tsm_run: the HPE estimator needs every lattice extent >= 4 (its exact orders)");
  // time-diluted sources (Sec. 2.3): noise on the slices t = t0 (mod dt) only, contracted there only
  Slices S = all_slices(c->dims[3]);
  if (prm->tdil_dt != 0) {
    const int T = c->dims[3];
    if (prm->tdil_dt < 1 || prm->tdil_dt > T || prm->tdil_t0 < 0 || prm->tdil_t0 >= prm->tdil_dt)
      return fail(c, DL_ERR_ARG, "dl_tsm_run: time dilution needs 1 <= tdil_dt <= T and 0 <= tdil_t0 < tdil_dt");
    if (prm->with_deriv)
      return fail(c, DL_ERR_ARG, "dl_tsm_run: time-diluted sources are contracted into local loops only");
    S = Slices{prm->tdil_t0, prm->tdil_dt, (T - 1 - prm->tdil_t0) / prm->tdil_dt + 1};
  }
  if ((s = enter(c)) != DL_OK) return s;
  auto t_all = std::chrono::steady_clock::now();
  if (c->profiling) c->prof_pending[0] = c->prof_pending[1] = c->prof_pending[2] = 1;
  if ((s = ensure_momenta(c, prm->p2max)) != DL_OK) return s;
  const int np = c->np, nd = prm->with_deriv ? 5 : 1, T = c->dims[3];
  // estimators: one-end, generalised one-end (and HPE); for time-diluted sources the
  // standard estimator (and HPE): the one-end trick sums over every sink time of one
  // source and does not restrict to the source's slices
  const bool tdil = prm->tdil_dt != 0;
  const int n_est = tdil ? (prm->hpe ? 2 : 1) : (prm->hpe ? 3 : 2);
  int est_mode[3] = {DL_EST_ONE_END, DL_EST_GEN, DL_EST_HPE};
  if (tdil) {
    est_mode[0] = DL_EST_STANDARD;
    est_mode[1] = DL_EST_HPE;
  }
  const long long per = (long long)T * np * nd * 16;
  // block = 0: buffers for the largest candidate until the autotuner has chosen
  const bool tune = prm->block == 0;
  int blk = tune ? DL_MAX_RHS : prm->block;
  double2 *acc_d, *acc_l, *bl, *bh, *res;
  double *obs1, *obs2;
  void* p;
  if ((s = ensure_buf(c, "ts_accd", sizeof(double2) * n_est * per, &p)) != DL_OK) return s;
  acc_d = (double2*)p;
  if ((s = ensure_buf(c, "ts_accl", sizeof(double2) * n_est * per, &p)) != DL_OK) return s;
  acc_l = (double2*)p;
  if ((s = ensure_buf(c, "ts_bl", sizeof(double2) * n_est * per * blk, &p)) != DL_OK) return s;
  bl = (double2*)p;
  if ((s = ensure_buf(c, "ts_bh", sizeof(double2) * n_est * per * blk, &p)) != DL_OK) return s;
  bh = (double2*)p;
  if ((s = ensure_buf(c, "ts_res", sizeof(double2) * n_est * per, &p)) != DL_OK) return s;
  res = (double2*)p;
  if ((s = ensure_buf(c, "ts_obs1", sizeof(double) * 4 * blk, &p)) != DL_OK) return s;
  obs1 = (double*)p;
  if ((s = ensure_buf(c, "ts_obs2", sizeof(double) * 4 * blk, &p)) != DL_OK) return s;
  obs2 = (double*)p;
  CK(cudaMemsetAsync(acc_d, 0, sizeof(double2) * n_est * per, c->st));
  CK(cudaMemsetAsync(acc_l, 0, sizeof(double2) * n_est * per, c->st));
  int ip0 = 0;
  {
    std::vector<int> lst(3 * np);
    int cnt;
    dl_momenta(prm->p2max, &cnt, lst.data());
    for (int k = 0; k < np; ++k)
      if (lst[3 * k] == 0 && lst[3 * k + 1] == 0 && lst[3 * k + 2] == 0) ip0 = k;
  }
  const double Ls = (double)c->dims[0] * c->dims[1] * c->dims[2];
  CK(dl::hpe_exact(c->kappa, c->amu, 1, c->misc, c->st));
  dl_tsm_info inf;
  memset(&inf, 0, sizeof(inf));
  inf.np = np;
  inf.nd = nd;
  inf.n_est = n_est;
  double t_hp = 0, t_lp = 0, t_ct = 0;
  bool any_nc = false, any_bd = false;

  // one precision's pipeline: noise -> solve -> contractions into `out`
  auto run_block = [&](int n, uint64_t first, bool hp, double2* out, double* obs, dl_solve_stats* st) -> dl_status {
    const int hi = hp ? PDF : P32;
    dl_solve_params sp;
    sp.tol = hp ? prm->tol_hp : prm->tol_lp;
    sp.max_iter = prm->max_iter;
    sp.prec_hi = hi;
    sp.prec_lo = internal_prec(hp ? prm->prec_hp_lo : prm->prec_lp_lo);
    sp.delta = hp ? prm->delta_hp : 0.0;
    sp.flavour = 1;
    sp.chunk = prm->chunk > 0 ? prm->chunk : 16;
    Batch B = make_batch(c, n);
    dl_status s2;
    if ((s2 = ensure_partial(c, B)) != DL_OK) return s2;
    Field *ee, *eo, *xe, *po;
    const char* tag = hp ? "64" : "32";
    if ((s2 = ensure_field(c, std::string("ts_ee") + tag, hi, B, &ee)) ||
        (s2 = ensure_field(c, std::string("ts_eo") + tag, hi, B, &eo)) ||
        (s2 = ensure_field(c, std::string("ts_xe") + tag, hi, B, &xe)) ||
        (s2 = ensure_field(c, std::string("ts_po") + tag, hi, B, &po)))
      return s2;
    CK(dl::noise_z4(B, hi, 0, ee->ref(), prm->seed, first, 0, c->st, S));
    CK(dl::noise_z4(B, hi, 1, eo->ref(), prm->seed, first, 0, c->st, S));
    bool guess = false;
    if (hp && prm->hp_guess) {  // start from the LP solution of the same noise (same block, FP32 field)
      Field* lp_xe;
      if ((s2 = ensure_field(c, "ts_xe32", P32, B, &lp_xe)) != DL_OK) return s2;
      CK(dl::copy(B, hi, P32, xe->ref(), lp_xe->ref(), nullptr, c->st));
      guess = true;
    }
    auto t0 = std::chrono::steady_clock::now();
    dl_status rs = (!hp && prm->lp_net) ? nn_map_block(prm->lp_net, c, B, ee, eo, xe, po)
                                        : solve_internal(c, B, sp, ee, eo, xe, po, false, st, guess);
    if (rs < 0) return rs;
    if (rs == DL_NOT_CONVERGED) any_nc = true;
    // an HP solve that broke down misses its tolerance and would bias Eq. estiTSM; an LP
    // solve keeps its last iterate, a valid (if poorer) LP map: the estimate stays unbiased
    if (rs == DL_BREAKDOWN && hp) any_bd = true;
    CK(cudaStreamSynchronize(c->st));
    auto t1 = std::chrono::steady_clock::now();
    (hp ? t_hp : t_lp) += std::chrono::duration<double>(t1 - t0).count();
    for (int e = 0; e < n_est; ++e) {
      double2* o = out + (size_t)e * per * blk;
      if (est_mode[e] == DL_EST_HPE && hp && prm->hpe_diff) {
        // the HPE estimator is linear in s: its HP-LP correction is eta^+ X (BH)^4 (s_HP - s_LP),
        // with the difference taken in double-float and (BH)^4 applied to it in FP32
        Field *lxe, *lxo, *de, *dd, *e3, *o3, *we, *wo;
        if ((s2 = ensure_field(c, "ts_xe32", P32, B, &lxe)) || (s2 = ensure_field(c, "ts_po32", P32, B, &lxo)) ||
            (s2 = ensure_field(c, "ts_hde", P32, B, &de)) || (s2 = ensure_field(c, "ts_hdo", P32, B, &dd)) ||
            (s2 = ensure_field(c, "ts_hee", P32, B, &e3)) || (s2 = ensure_field(c, "ts_heo", P32, B, &o3)))
          return s2;
        CK(dl::diff(B, P32, hi, P32, de->ref(), xe->ref(), lxe->ref(), c->st));
        CK(dl::diff(B, P32, hi, P32, dd->ref(), po->ref(), lxo->ref(), c->st));
        CK(dl::copy(B, P32, hi, e3->ref(), ee->ref(), nullptr, c->st));
        CK(dl::copy(B, P32, hi, o3->ref(), eo->ref(), nullptr, c->st));
        if ((s2 = bh_power(c, B, P32, 1, 4, de, dd, &we, &wo)) != DL_OK) return s2;
        if ((s2 = contract_internal(c, B, P32, DL_EST_HPE, 0, prm->p2max, we, wo, e3, o3, 1.0, 0.0, o, 0, S)) != DL_OK)
          return s2;
      } else if (est_mode[e] == DL_EST_HPE) {
        Field *we, *wo;
        if ((s2 = bh_power(c, B, hi, 1, 4, xe, po, &we, &wo)) != DL_OK) return s2;
        if ((s2 = contract_internal(c, B, hi, DL_EST_HPE, 0, prm->p2max, we, wo, ee, eo, 1.0, 0.0, o, 0, S)) != DL_OK)
          return s2;
        CK(dl::add_exact_p0(B, np, nd, ip0, c->misc, Ls, o, S, c->st));
      } else {
        double pr = 1.0, pi = 0.0;  // the estimator's factor (Eqs. loopSt, loopVv, loopStD)
        if (est_mode[e] == DL_EST_ONE_END) {
          pr = 0.0;
          pi = -4.0 * c->kappa * c->amu;
        } else if (est_mode[e] == DL_EST_GEN) {
          pr = 2.0;
        }
        if ((s2 = contract_internal(c, B, hi, est_mode[e], prm->with_deriv, prm->p2max, xe, po, ee, eo, pr, pi, o, 0, S)) !=
            DL_OK)
          return s2;
      }
    }
    // per-noise observables: i g5 and g_z g5 loops (one-end and generalised; both from
    // the standard estimator for time-diluted sources)
    CK(dl::observables(out, tdil ? out : out + (size_t)per * blk, n, T, np, nd, ip0, obs, c->st));
    CK(cudaStreamSynchronize(c->st));
    t_ct += std::chrono::duration<double>(std::chrono::steady_clock::now() - t1).count();
    return rs;
  };

  if (tune) {
    const std::vector<int> key{prm->prec_lp_lo, prm->p2max, prm->with_deriv, prm->hpe, prm->tdil_dt, prm->tdil_t0};
    auto it = c->tsm_blocks.find(key);
    if (it != c->tsm_blocks.end()) {
      blk = it->second;
    } else {
      // one LP block per candidate on noise indices from 2^32 (outside any workload's),
      // once untimed (CUDA graphs, buffers) and once timed; least time per right-hand side
      const auto tt0 = std::chrono::steady_clock::now();
      const double sv_hp = t_hp, sv_lp = t_lp, sv_ct = t_ct;
      const bool sv_nc = any_nc, sv_bd = any_bd;
      int best_b = 16;
      double best = 1e300;
      for (int cand : {8, 16, 32}) {
        if (cand > DL_MAX_RHS) continue;
        double dt = 0.0;
        for (int rep = 0; rep < 2; ++rep) {
          dl_solve_stats st;
          memset(&st, 0, sizeof(st));
          CK(cudaStreamSynchronize(c->st));
          const auto a0 = std::chrono::steady_clock::now();
          if ((s = run_block(cand, (uint64_t)1 << 32, false, bl, obs1, &st)) < 0) return s;
          CK(cudaStreamSynchronize(c->st));
          dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - a0).count();
        }
        if (dt / cand < best) {
          best = dt / cand;
          best_b = cand;
        }
      }
      t_hp = sv_hp;
      t_lp = sv_lp;
      t_ct = sv_ct;
      any_nc = sv_nc;
      any_bd = sv_bd;
      blk = best_b;
      c->tsm_blocks[key] = blk;
      inf.seconds_tune = std::chrono::duration<double>(std::chrono::steady_clock::now() - tt0).count();
    }
  }
  inf.block = blk;
  std::vector<double> hbuf(4 * blk);
  for (int b0 = 0; b0 < prm->n_hp; b0 += blk) {
    int n = std::min(blk, prm->n_hp - b0);
    dl_solve_stats st;
    memset(&st, 0, sizeof(st));
    if ((s = run_block(n, (uint64_t)b0, false, bl, obs1, &st)) < 0) return s;
    for (int i = 0; i < n; ++i) inf.iters_lp += st.iters[i];
    memset(&st, 0, sizeof(st));
    if ((s = run_block(n, (uint64_t)b0, true, bh, obs2, &st)) < 0) return s;
    for (int i = 0; i < n; ++i) inf.iters_hp += st.iters[i];
    for (int e = 0; e < n_est; ++e) {
      // with hpe_diff the HP block already holds the HPE correction itself
      const bool direct = est_mode[e] == DL_EST_HPE && prm->hpe_diff;
      CK(dl::col_accumulate(bh + (size_t)e * per * blk, direct ? nullptr : bl + (size_t)e * per * blk, n, per, 1.0,
                            acc_d + (size_t)e * per, c->st));
    }
    if (obs_lp_pair) {
      CK(cudaMemcpyAsync(hbuf.data(), obs1, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
      memcpy(obs_lp_pair + 4 * b0, hbuf.data(), sizeof(double) * 4 * n);
    }
    if (obs_hp) {
      CK(cudaMemcpyAsync(hbuf.data(), obs2, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
      memcpy(obs_hp + 4 * b0, hbuf.data(), sizeof(double) * 4 * n);
    }
  }
  for (int b0 = 0; b0 < prm->n_lp; b0 += blk) {
    int n = std::min(blk, prm->n_lp - b0);
    dl_solve_stats st;
    memset(&st, 0, sizeof(st));
    if ((s = run_block(n, (uint64_t)(prm->n_hp + b0), false, bl, obs1, &st)) < 0) return s;
    for (int i = 0; i < n; ++i) inf.iters_lp += st.iters[i];
    for (int e = 0; e < n_est; ++e)
      CK(dl::col_accumulate(bl + (size_t)e * per * blk, nullptr, n, per, 1.0, acc_l + (size_t)e * per, c->st));
    if (obs_lp) {
      CK(cudaMemcpyAsync(hbuf.data(), obs1, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
      memcpy(obs_lp + 4 * b0, hbuf.data(), sizeof(double) * 4 * n);
    }
  }
  // Eq. estiTSM: mean HP-LP correction + mean over the fresh LP set
  const double a = prm->n_hp > 0 ? 1.0 / prm->n_hp : 0.0, b = prm->n_lp > 0 ? 1.0 / prm->n_lp : 0.0;
  CK(dl::combine(acc_d, acc_l, a, b, (long long)n_est * per, res, c->st));
  if (loops) CK(cudaMemcpyAsync(loops, res, sizeof(double2) * n_est * per, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  inf.seconds_total = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_all).count();
  inf.seconds_hp = t_hp;
  inf.seconds_lp = t_lp;
  inf.seconds_contract = t_ct;
  if (info) {
    inf.not_converged = (any_nc || any_bd) ? 1 : 0;
    *info = inf;
  }
  if ((s = leave(c)) != DL_OK) return s;
  if (any_bd) return fail(c, DL_BREAKDOWN, "an HP solve of the TSM broke down (its loops are not valid)");
  return any_nc ? fail(c, DL_NOT_CONVERGED, "a TSM solve hit max_iter") : DL_OK;
} DL_CATCH(c)

dl_status dl_batch_loops(dl_ctx* c, const dl_batch_params* prm, double* loops, void* sol, dl_batch_info* info) try {
  if (!c || !prm) return DL_ERR_ARG;
  const int nl = (int)c->lats.size();
  for (auto& L : c->lats)
    if (!L.has_gauge) return fail(c, DL_ERR_STATE, "dl_batch_loops: a lattice has no gauge field");
  const int n = prm->n;
  if (n < 1 || n * nl > DL_NCMAX || !(prm->tol > 0.0) || prm->max_iter < 1 ||
      !(prm->prec_hi == DL_F64 || prm->prec_hi == DL_F32) || prm->prec_lo < prm->prec_hi || prm->prec_lo > DL_F16 ||
      prm->delta < 0.0 || prm->delta >= 1.0 ||
      !(prm->tile == 0 || prm->tile == 4 || prm->tile == 8 || prm->tile == 16 || prm->tile == 32))
    return fail(c, DL_ERR_ARG, "dl_batch_loops: bad parameters");
  dl_status s;
  if ((s = enter(c)) != DL_OK) return s;
  const int hi = internal_prec(prm->prec_hi);
  dl_batch_info inf;
  memset(&inf, 0, sizeof(inf));
  auto t0 = std::chrono::steady_clock::now();
  // noise, source preparation and solve for every lattice in one batch
  auto run = [&](int tile, int max_iter, double tol, double delta, Batch& B, Field** fe, bool* nc) -> dl_status {
    if (!make_batch_multi(c, tile, n, B)) return fail(c, DL_ERR_ARG, "dl_batch_loops: too many instances for the tile");
    dl_status s2;
    Field *ee, *eo, *xe, *po;
    if ((s2 = ensure_field(c, "bt_ee", hi, B, &ee)) || (s2 = ensure_field(c, "bt_eo", hi, B, &eo)) ||
        (s2 = ensure_field(c, "bt_xe", hi, B, &xe)) || (s2 = ensure_field(c, "bt_po", hi, B, &po)))
      return s2;
    CK(dl::noise_z4(B, hi, 0, ee->ref(), prm->seed, 0, 0, c->st));
    CK(dl::noise_z4(B, hi, 1, eo->ref(), prm->seed, 0, 0, c->st));
    dl_solve_params sp;
    sp.tol = tol;
    sp.max_iter = max_iter;
    sp.prec_hi = hi;
    sp.prec_lo = internal_prec(prm->prec_lo);
    sp.delta = delta;
    sp.flavour = 1;
    sp.chunk = 0;
    dl_status rs = solve_internal(c, B, sp, ee, eo, xe, po, false, nullptr);
    if (rs < 0) return rs;
    if (nc) *nc = rs == DL_NOT_CONVERGED || rs == DL_BREAKDOWN;
    fe[0] = ee;
    fe[1] = eo;
    fe[2] = xe;
    fe[3] = po;
    return DL_OK;
  };
  // right-hand-side tile: given, or the fastest per column-iteration of a short timed run
  int tile = prm->tile;
  if (tile == 0) {
    double best = 1e300;
    const int cand[3] = {8, 16, 32};
    for (int ci = 0; ci < 3; ++ci) {
      Batch B;
      Field* fe[4];
      if (!make_batch_multi(c, cand[ci], n, B)) continue;
      if ((s = run(cand[ci], 2, 1e-300, 0.0, B, fe, nullptr)) != DL_OK) return s;  // capture the graph
      CK(cudaStreamSynchronize(c->st));
      auto a0 = std::chrono::steady_clock::now();
      if ((s = run(cand[ci], 6, 1e-300, 0.0, B, fe, nullptr)) != DL_OK) return s;
      CK(cudaStreamSynchronize(c->st));
      const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - a0).count();
      if (dt < best) {
        best = dt;
        tile = cand[ci];
      }
    }
    if (tile == 0) return fail(c, DL_ERR_ARG, "dl_batch_loops: no tile fits");
  }
  auto t1 = std::chrono::steady_clock::now();
  Batch B;
  Field* fe[4];
  bool nc = false;
  if ((s = run(tile, prm->max_iter, prm->tol, prm->delta, B, fe, &nc)) != DL_OK) return s;
  CK(cudaStreamSynchronize(c->st));
  auto t2 = std::chrono::steady_clock::now();
  // loops at p = 0 per lattice: [2 estimators][n][T_l][4][4]
  if ((s = ensure_momenta(c, 0)) != DL_OK) return s;
  size_t total = 0;
  std::vector<size_t> loff(nl), soff(nl);
  size_t so = 0;
  for (int l = 0; l < nl; ++l) {
    loff[l] = total;
    total += (size_t)2 * n * c->lats[l].dims[3] * 16;
    soff[l] = so;
    so += (size_t)n * 2 * c->lats[l].Vh * 12;
  }
  void* p;
  if ((s = ensure_buf(c, "bt_loops", sizeof(double2) * total, &p)) != DL_OK) return s;
  double2* dloops = (double2*)p;
  int inst = 0;
  for (int l = 0; l < nl; ++l)
    for (int k = 0; k * tile < n; ++k, ++inst) {
      Batch B1;
      memset(&B1, 0, sizeof(B1));
      B1.nlat = 1;
      B1.lat[0] = B.lat[inst];
      B1.pstride = B.pstride;
      dl::blocks_for(B1, 256);
      const int T = B1.lat[0].T;
      double2* o1 = dloops + loff[l] + ((size_t)0 * n + (size_t)k * tile) * T * 16;
      double2* o2 = dloops + loff[l] + ((size_t)1 * n + (size_t)k * tile) * T * 16;
      const double pim = -4.0 * B1.lat[0].kappa * B1.lat[0].amu;
      if ((s = contract_internal(c, B1, hi, DL_EST_ONE_END, 0, 0, fe[2], fe[3], fe[0], fe[1], 0.0, pim, o1, 0)) != DL_OK)
        return s;
      if ((s = contract_internal(c, B1, hi, DL_EST_GEN, 0, 0, fe[2], fe[3], fe[0], fe[1], 2.0, 0.0, o2, 0)) != DL_OK)
        return s;
      if (sol) {
        double2* sl = (double2*)sol + soff[l] + (size_t)k * tile * 2 * B1.lat[0].Vh * 12;
        CK(dl::unpack(B1, hi, 0, sl, fe[2]->ref(), DL_C128, c->st));
        CK(dl::unpack(B1, hi, 1, sl, fe[3]->ref(), DL_C128, c->st));
      }
    }
  if (loops) CK(cudaMemcpyAsync(loops, dloops, sizeof(double2) * total, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  auto t3 = std::chrono::steady_clock::now();
  inf.tile = tile;
  inf.instances = B.nlat;
  inf.seconds_tune = std::chrono::duration<double>(t1 - t0).count();
  inf.seconds_solve = std::chrono::duration<double>(t2 - t1).count();
  inf.seconds_contract = std::chrono::duration<double>(t3 - t2).count();
  inf.not_converged = nc ? 1 : 0;
  for (int l = 0; l < nl && l < DL_MAX_LAT; ++l) {
    int mx = 0;
    double rmax = 0.0;
    for (int i = 0; i < n; ++i) {
      const int gc = l * n + i;  // instances of a lattice are consecutive, columns in order
      if (gc < (int)c->last_iters.size()) mx = std::max(mx, c->last_iters[gc]);
      if (gc < (int)c->last_resid.size()) rmax = std::max(rmax, c->last_resid[gc]);
    }
    inf.iters_max[l] = mx;
    inf.resid_max[l] = rmax;
  }
  if (info) *info = inf;
  if ((s = leave(c)) != DL_OK) return s;
  return nc ? fail(c, DL_NOT_CONVERGED, "dl_batch_loops: a solve hit max_iter") : DL_OK;
} DL_CATCH(c)

}  // extern "C"

// ============================================================================
// Allocation-free operator application.
//
// Some callers cannot allocate device memory when they apply an operator: a
// host framework whose caching allocator already owns all device memory, a
// latency-critical loop that must not wait for cudaMalloc's implicit device
// synchronisation, or code that runs after its memory budget is fixed.  For
// them dl_apply_noalloc does what dl_apply does, but its working fields live in
// one file-scope device array of DL_NOALLOC_BYTES instead of the context's
// workspace.  The array exists on every GPU that loads this library, for the
// lifetime of the process.
#define DL_NOALLOC_BYTES (64ull << 20)
static __device__ __align__(256) unsigned char g_noalloc_scratch[DL_NOALLOC_BYTES];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[256] = {nullptr};

// Device address of the scratch array on the current device; looked up once
// per device (the first call on a device does this, so it should come before
// any stream capture).  In host code the array's name is only a stand-in.
cudaError_t noalloc_scratch(int dev, unsigned char** out) {
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = (unsigned char*)g_noalloc_ptr[dev];
  return cudaSuccess;
}
}  // namespace

extern "C" dl_status dl_apply_noalloc(dl_ctx* c, int op, int prec, int f, int n, const void* in, const void* aux,
                                      void* out, int dtype) try {
  dl_status s;
  if ((s = check_ctx(c, true)) != DL_OK) return s;
  if (!in || !out || n < 1 || n > DL_MAX_RHS || (f != 1 && f != -1) || prec_rank(prec) < 0 ||
      (dtype != DL_C128 && dtype != DL_C64) || op < DL_OP_M || op > DL_OP_BH)
    return fail(c, DL_ERR_ARG, "dl_apply_noalloc: bad argument");
  if (op == DL_OP_RECON && !aux) return fail(c, DL_ERR_ARG, "DL_OP_RECON needs aux");
  prec = internal_prec(prec);
  // seven parity fields (in, out, aux for both parities, one temporary), each
  // 256-byte aligned, must fit the fixed array
  const size_t items = (size_t)c->Vh << ilog2ceil(n);
  const size_t data_b = (items * chunk_bytes(prec) + 255) & ~(size_t)255;
  const size_t norm_b = prec == P16 ? ((items * sizeof(float) + 255) & ~(size_t)255) : 0;
  const size_t need = 7 * (data_b + norm_b);
  if (need > DL_NOALLOC_BYTES) {
    char msg[200];
    snprintf(msg, sizeof(msg), "dl_apply_noalloc: %zu bytes of working fields exceed the %llu-byte fixed scratch", need,
             (unsigned long long)DL_NOALLOC_BYTES);
    return fail(c, DL_ERR_ARG, msg);
  }
  if ((s = enter(c)) != DL_OK) return s;
  unsigned char* base = nullptr;
  CK(noalloc_scratch(c->dev, &base));
  FieldRef fr[7];
  for (int k = 0; k < 7; ++k) {
    unsigned char* p = base + (size_t)k * (data_b + norm_b);
    fr[k] = FieldRef{p, prec == P16 ? (float*)(p + data_b) : nullptr};
  }
  const FieldRef ie = fr[0], io = fr[1], oe = fr[2], oo = fr[3], ae = fr[4], ao = fr[5], t = fr[6];
  Batch B = make_batch(c, n);
  CK(dl::pack(B, prec, 0, ie, in, dtype, c->st));
  CK(dl::pack(B, prec, 1, io, in, dtype, c->st));
  if (aux) {
    CK(dl::pack(B, prec, 0, ae, aux, dtype, c->st));
    CK(dl::pack(B, prec, 1, ao, aux, dtype, c->st));
  }
  GaugeSet g{c->g64, c->g32, c->g16, c->gdf};
  const int gr = grec_of(c, prec);
  auto D = [&](int epi_kind, bool dag, int par, FieldRef src, FieldRef ax, FieldRef dst, const EpiSet& E) {
    return dl::dslash(B, prec, gr, epi_kind, dag, par, src, ax, dst, g, E, nullptr, nullptr, NOF, NOF, NOF, nullptr,
                      c->st);
  };
  switch (op) {
    case DL_OP_M:
    case DL_OP_MDAG: {
      const bool dag = op == DL_OP_MDAG;
      EpiSet E = epiB(B, CK_MK, 0, 0, 1, dag ? -f : f);
      CK(D(EPI_AUX, dag, 0, io, ie, oe, E));
      CK(D(EPI_AUX, dag, 1, ie, io, oo, E));
      break;
    }
    case DL_OP_HOP: {
      EpiSet E = epiB(B, CK_ONE, 0, 0, 0, 0);
      CK(D(EPI_PLAIN, false, 0, io, NOF, oe, E));
      CK(D(EPI_PLAIN, false, 1, ie, NOF, oo, E));
      break;
    }
    case DL_OP_MHAT:
    case DL_OP_MHAT_DAG: {
      const bool dag = op == DL_OP_MHAT_DAG;
      CK(stage1(c, B, prec, dag, f, ie, t, nullptr));
      CK(stage2(c, B, prec, dag, f, t, ie, oe, nullptr, nullptr));
      CK(dl::zero(B, prec, oo, nullptr, c->st));
      break;
    }
    case DL_OP_PREP: {
      EpiSet Ei = epiB(B, CK_ONE, 2, f, 0, 0);
      CK(dl::twist(B, prec, t, io, Ei, nullptr, c->st));
      EpiSet E = epiB(B, CK_K, 0, 0, 0, 0);
      CK(D(EPI_AUX, false, 0, t, ie, oe, E));
      CK(dl::zero(B, prec, oo, nullptr, c->st));
      break;
    }
    case DL_OP_RECON: {
      CK(dl::copy(B, prec, prec, oe, ie, nullptr, c->st));
      EpiSet E = epiB(B, CK_K, 2, f, 0, 0);
      CK(D(EPI_AUX, false, 1, ie, ao, oo, E));
      break;
    }
    case DL_OP_BH: {
      EpiSet E = epiB(B, CK_MK, 2, f, 0, 0);
      CK(D(EPI_PLAIN, false, 0, io, NOF, oe, E));
      CK(D(EPI_PLAIN, false, 1, ie, NOF, oo, E));
      break;
    }
  }
  CK(dl::unpack(B, prec, 0, out, oe, dtype, c->st));
  CK(dl::unpack(B, prec, 1, out, oo, dtype, c->st));
  return leave(c);
} DL_CATCH(c)
