// Host-side state shared by the translation units of the C ABI: the context
// object, its device workspaces and the helpers that build batches, epilogues
// and fields.  Not part of the public interface (include/discloop.h is).
#pragma once

#include <map>
#include <new>
#include <string>
#include <vector>

#include "discloop.h"
#include "dl_kernels.h"

struct Field {
  int prec = -1;
  size_t items = 0;
  void* data = nullptr;
  float* norm = nullptr;
  FieldRef ref() const { return FieldRef{data, norm}; }
};

struct GraphEntry {
  std::string key;
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;  // kernel nodes in the graph
  dl::StencilTally tally;  // stencil launches of one replay of the body, by class
};

inline int ilog2ceil(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

inline size_t chunk_bytes(int prec) { return (prec == P64 || prec == PDF) ? 192 : (prec == P32 ? 96 : 48); }

// The API's FP64 precision as the kernels run it: double-float arithmetic on
// FP32 units (dl_df.cuh), since GB300's FP64 rate is a small fraction of FP32.
inline int internal_prec(int api_prec) {
  return api_prec == DL_F64 ? PDF : (api_prec == DL_F64_IEEE ? P64 : api_prec);
}
// 0 for both FP64 forms, 1 FP32, 2 16-bit; -1 for anything else
inline int prec_rank(int api_prec) {
  return (api_prec == DL_F64 || api_prec == DL_F64_IEEE) ? 0 : (api_prec == DL_F32 ? 1 : (api_prec == DL_F16 ? 2 : -1));
}

struct LatInfo {
  int dims[4];
  int Vh;
  double kappa = 0.125, amu = 0.0, tbc = -1.0;
  long long gsite_off = 0;  // parity-site offset of this lattice in the gauge arrays
  bool has_gauge = false;
};

struct dl_ctx {
  std::vector<LatInfo> lats;  // one entry for dl_create, several for dl_create_multi
  // TSM blocks chosen by the autotuner: (LP precision, p2max, derivative, HPE, tdil_dt, tdil_t0) -> block
  std::map<std::vector<int>, int> tsm_blocks;
  long long Vh_total = 0;
  int dev = 0;
  cudaStream_t st = nullptr;    // internal stream (non-blocking; capturable)
  cudaStream_t user = nullptr;  // caller's stream
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int dims[4] = {0, 0, 0, 0};
  int Vh = 0;
  double kappa = 0.125, amu = 0.0, tbc = -1.0;
  int rec32 = 12, rec16 = 8;
  void* g64 = nullptr;
  void* gdf = nullptr;  // double-float copy of the FP64 links (same layout, 144 B per link)
  void* g32 = nullptr;
  void* g16 = nullptr;
  bool has_gauge = false;
  std::string err;
  std::map<std::string, Field> ws;
  double* partial = nullptr;
  size_t partial_blocks = 0;
  int* loopctr = nullptr;  // iterations run by the current graph launch, its limit, host-loop flag
  bool use_graphs = true;  // CG loop as a conditional CUDA graph (DL_GRAPHS=0: host loop)
  int* waitc = nullptr;    // per column: iterations spent waiting for a reliable update
  double* S = nullptr;  // [DL_NS][DL_NCMAX]
  int* active = nullptr;
  int* flags = nullptr;
  int* iters = nullptr;
  int* upd = nullptr;
  int* all = nullptr;  // all-ones mask
  double2* misc = nullptr;  // small complex scratch (HPE exact part, observables)
  int* mom = nullptr;
  int mom_p2 = -1, np = 0;
  void* scratch = nullptr;  // contraction scratch
  size_t scratch_bytes = 0;
  std::map<std::string, DevBuf> bufs;
  std::vector<GraphEntry> graphs;
  std::vector<int> last_iters;        // per column, last solve
  std::vector<double> last_resid;     // per column, last solve
  // live stencil timing: events around the four operator launches of the first
  // CG iteration of every captured chunk; sums per (stage, precision)
  int profiling = 0;
  int prof_pending[3] = {0, 0, 0};  // take one stencil sample per precision when set
  cudaEvent_t pev[8] = {nullptr};
  double prof_ms[4][3] = {{0}};
  long long prof_n[4][3] = {{0}};
  long long prof_items[4][3] = {{0}};  // site-column items processed, summed over sampled launches
};

#define CK(expr)                                                   \
  do {                                                             \
    cudaError_t _e = (expr);                                       \
    if (_e != cudaSuccess) return cuda_fail(c, _e, #expr);         \
  } while (0)

namespace dlh {

// Epilogue coefficient kinds, evaluated per lattice of a batch.
enum { CK_ONE = 0, CK_K = 1, CK_MK = 2, CK_MK2 = 3 };  // 1, kappa, -kappa, -kappa^2

extern const FieldRef NOF;

dl_status fail(dl_ctx* c, dl_status s, const std::string& m);
dl_status cuda_fail(dl_ctx* c, cudaError_t e, const char* what);
Batch make_batch(const dl_ctx* c, int ncol);
EpiSet epiB(const Batch& B, int ck, int t1, int f1, int t2, int f2);
int grec_of(const dl_ctx* c, int prec);
dl_status ensure_field(dl_ctx* c, const std::string& base, int prec, const Batch& B, Field** out);
dl_status ensure_partial(dl_ctx* c, const Batch& B);
dl_status ensure_buf(dl_ctx* c, const std::string& name, size_t bytes, void** out);
dl_status enter(dl_ctx* c);
dl_status leave(dl_ctx* c);
dl_status check_ctx(dl_ctx* c, bool need_gauge);
cudaError_t colsum(dl_ctx* c, const Batch& B, int slot);
// x = N(eta) column by column with the learned map (FP32 fields of a single-lattice block)
dl_status nn_map_block(dl_nn* nn, dl_ctx* c, const Batch& B, Field* ee, Field* eo, Field* xe, Field* xo);

// An exception raised by host-side bookkeeping inside an entry point (a failed host
// allocation in a std::vector, std::map or std::string) becomes a status and a
// message; nothing is thrown across the C boundary.
inline dl_status host_exception(dl_ctx* c, dl_status s) noexcept {
  if (c) {
    try {
      c->err = s == DL_ERR_OOM ? "host allocation failed" : "unexpected host exception";
    } catch (...) {
    }
  }
  return s;
}

}  // namespace dlh

// Handler of the function-try-block around the body of every entry point.
#define DL_CATCH(ctx_expr)                                                   \
  catch (const std::bad_alloc&) {                                           \
    return dlh::host_exception((ctx_expr), DL_ERR_OOM);                     \
  }                                                                          \
  catch (...) {                                                              \
    return dlh::host_exception((ctx_expr), DL_ERR_STATE);                   \
  }
