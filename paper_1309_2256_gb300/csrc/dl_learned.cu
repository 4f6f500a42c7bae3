// Host side of the learned preconditioner (no counterpart in the paper): the
// network object, its inference, loss and gradient, Adam training, the flexible
// GCR solver that uses it, and the map that stands in for low-precision solves
// in the truncated solver method.  Every arithmetic step runs in the kernels of
// dl_network.cu, dl_dslash.cu and dl_blas.cu; this file orders launches and
// reads back scalars.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "dl_host.h"

struct dl_nn {
  dl_ctx* c = nullptr;
  int nl = 0, C = 0, act = P32;
  std::vector<int> ci, co;
  std::vector<size_t> woff, poff;  // complex offsets of each layer's weights / weight-gradient partials
  size_t nw = 0, npart = 0;
  float2 *W = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr, *wpart = nullptr;
  int slots = 0;   // persistent CTAs of the weight-gradient kernel (one partial slot each)
  int adam_t = 0;  // Adam steps taken
  double* dscal = nullptr;  // device scalars: [0, 2) dot products, [2, 2 + 2 * nloss) loss partial sums
  int nloss = 0;
  // tensor-core layers (bfloat16 activations): per layer 36 B chunks of 2 KB laid out from W
  // (tcB) and from the adjoint layer's weights (tcBa, for input gradients and N^+)
  bool use_tc = false;
  bool tc_dirty = true;     // W changed since the chunks were laid out
  void* tcB = nullptr;
  void* tcBa = nullptr;
  float2* Wa = nullptr;     // one layer's adjoint weights (scratch, 36 x 16 x 16 complex)
  int* tc_err = nullptr;    // set by the kernel when a bounded wait ran out
};

using namespace dlh;

namespace {

constexpr int NN_MAX_LAYERS = 16;

int lg_in(const dl_nn* nn, int l) { return l == 0 ? 0 : ilog2ceil(nn->C); }
int lg_out(const dl_nn* nn, int l) { return l == nn->nl - 1 ? 0 : ilog2ceil(nn->C); }

size_t site_bytes(int dtype) { return dtype == DL_C128 ? 12 * 16 : 12 * 8; }

// Activation (tag "x") or gradient (tag "g") fields of layer input l = 0..nl, both parities.
dl_status act_fields(dl_nn* nn, const char* tag, int l, Field** e, Field** o) {
  dl_ctx* c = nn->c;
  const int ch = (l == 0 || l == nn->nl) ? 1 : nn->C;
  const Batch B = make_batch(c, ch);
  const std::string b = std::string("nn_") + tag + std::to_string(l);
  dl_status s;
  if ((s = ensure_field(c, b + "e", nn->act, B, e)) || (s = ensure_field(c, b + "o", nn->act, B, o))) return s;
  return DL_OK;
}

struct Acts {
  Field* e[NN_MAX_LAYERS + 1];
  Field* o[NN_MAX_LAYERS + 1];
};

dl_status get_acts(dl_nn* nn, const char* tag, int l0, Acts& A) {
  dl_status s;
  for (int l = l0; l <= nn->nl; ++l)
    if ((s = act_fields(nn, tag, l, &A.e[l], &A.o[l])) != DL_OK) return s;
  return DL_OK;
}

constexpr size_t TC_LAYER_BYTES = 36 * 2048;

// Lay out the tensor-core B chunks of every layer and of its adjoint after W changed.
dl_status tc_prepare(dl_nn* nn) {
  dl_ctx* c = nn->c;
  if (!nn->use_tc || !nn->tc_dirty) return DL_OK;
  for (int l = 0; l < nn->nl; ++l) {
    CK(dl::nn_tc_prep(nn->W + nn->woff[l], nn->ci[l], nn->co[l], (char*)nn->tcB + l * TC_LAYER_BYTES, c->st));
    CK(dl::nn_adj_weights(nn->W + nn->woff[l], nn->ci[l], nn->co[l], nn->Wa, c->st));
    CK(dl::nn_tc_prep(nn->Wa, nn->co[l], nn->ci[l], (char*)nn->tcBa + l * TC_LAYER_BYTES, c->st));
  }
  nn->tc_dirty = false;
  return DL_OK;
}

// G[l] = layer_l^+ (G[l+1]), output parity p: the adjoint layer on the tensor cores
// (bfloat16 activations, when enabled), else the input-gradient kernel on the CUDA cores.
dl_status layer_adjoint(dl_nn* nn, const LatDesc& L, int l, int p, const Acts& G) {
  dl_ctx* c = nn->c;
  FieldRef out = p ? G.o[l]->ref() : G.e[l]->ref();
  if (nn->use_tc)
    CK(dl::nn_forward_tc(L, c->rec32, p, G.e[l + 1]->ref(), G.o[l + 1]->ref(), out, c->g32,
                         (const char*)nn->tcBa + l * TC_LAYER_BYTES, nn->co[l], nn->ci[l], lg_out(nn, l), lg_in(nn, l),
                         nn->tc_err, c->st));
  else
    CK(dl::nn_backward_x(L, nn->act, c->rec32, p, G.e[l + 1]->ref(), G.o[l + 1]->ref(), out, c->g32,
                         nn->W + nn->woff[l], nn->ci[l], nn->co[l], lg_in(nn, l), lg_out(nn, l), c->st));
  return DL_OK;
}

// X[l+1] = layer_l(X[l]) for every layer, both output parities: on the tensor cores
// for bfloat16 activations (when enabled), else on the CUDA cores.
dl_status forward(dl_nn* nn, const Acts& X) {
  dl_ctx* c = nn->c;
  const LatDesc L = make_batch(c, 1).lat[0];
  dl_status st;
  if ((st = tc_prepare(nn)) != DL_OK) return st;
  for (int l = 0; l < nn->nl; ++l)
    for (int p = 0; p < 2; ++p) {
      FieldRef out = p ? X.o[l + 1]->ref() : X.e[l + 1]->ref();
      if (nn->use_tc)
        CK(dl::nn_forward_tc(L, c->rec32, p, X.e[l]->ref(), X.o[l]->ref(), out, c->g32,
                             (const char*)nn->tcB + l * TC_LAYER_BYTES, nn->ci[l], nn->co[l], lg_in(nn, l),
                             lg_out(nn, l), nn->tc_err, c->st));
      else
        CK(dl::nn_forward(L, nn->act, c->rec32, p, X.e[l]->ref(), X.o[l]->ref(), out, c->g32, nn->W + nn->woff[l],
                          nn->ci[l], nn->co[l], lg_in(nn, l), lg_out(nn, l), c->st));
    }
  return DL_OK;
}

// the tensor-core kernels' bounded waits: an expired wait is an error of the call
dl_status check_tc(dl_nn* nn) {
  dl_ctx* c = nn->c;
  if (!nn->use_tc) return DL_OK;
  int h = 0;
  CK(cudaMemcpyAsync(&h, nn->tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (h) return fail(c, DL_ERR_CUDA, "tensor-core forward: a bounded wait expired");
  return DL_OK;
}

// Gradient pass from G[nl] (already holding dL/d conj(y)): weight-gradient
// partials of every layer, input gradients of layers 1..nl-1.
dl_status backward(dl_nn* nn, const Acts& X, const Acts& G) {
  dl_ctx* c = nn->c;
  const LatDesc L = make_batch(c, 1).lat[0];
  dl_status st;
  if ((st = tc_prepare(nn)) != DL_OK) return st;
  for (int l = nn->nl - 1; l >= 0; --l) {
    for (int p = 0; p < 2; ++p) {
      FieldRef gp = p ? G.o[l + 1]->ref() : G.e[l + 1]->ref();
      if (nn->use_tc)
        CK(dl::nn_backward_w_tc(L, c->rec32, p, X.e[l]->ref(), X.o[l]->ref(), gp, c->g32, nn->ci[l], nn->co[l],
                                lg_in(nn, l), lg_out(nn, l), nn->wpart + nn->poff[l], nn->slots, nn->tc_err, c->st));
      else
        CK(dl::nn_backward_w(L, nn->act, c->rec32, p, X.e[l]->ref(), X.o[l]->ref(), gp, c->g32, nn->ci[l], nn->co[l],
                             lg_in(nn, l), lg_out(nn, l), nn->wpart + nn->poff[l], nn->slots, c->st));
    }
    if (l > 0)
      for (int p = 0; p < 2; ++p)
        if ((st = layer_adjoint(nn, L, l, p, G)) != DL_OK) return st;
  }
  return DL_OK;
}

// G[0] = N^+ G[nl]: the adjoint of every layer from the last to the first.
dl_status adjoint(dl_nn* nn, const Acts& G) {
  dl_ctx* c = nn->c;
  const LatDesc L = make_batch(c, 1).lat[0];
  dl_status st;
  if ((st = tc_prepare(nn)) != DL_OK) return st;
  for (int l = nn->nl - 1; l >= 0; --l)
    for (int p = 0; p < 2; ++p)
      if ((st = layer_adjoint(nn, L, l, p, G)) != DL_OK) return st;
  return DL_OK;
}

dl_status zero_wpart(dl_nn* nn) {
  dl_ctx* c = nn->c;
  CK(cudaMemsetAsync(nn->wpart, 0, sizeof(float2) * nn->npart * nn->slots, c->st));
  return DL_OK;
}

dl_status reduce_grad(dl_nn* nn) {
  dl_ctx* c = nn->c;
  for (int l = 0; l < nn->nl; ++l)
    CK(dl::nn_wsum(nn->wpart + nn->poff[l], nn->slots, (size_t)36 * nn->co[l] * nn->ci[l], nn->grad + nn->woff[l], c->st));
  return DL_OK;
}

// Pair k: eta_k into the network input, s_k into the FP32 loss targets
dl_status pack_pair(dl_nn* nn, const void* eta, const void* s, int dtype, int k, const Acts& X, Field* se, Field* so) {
  dl_ctx* c = nn->c;
  const Batch B1 = make_batch(c, 1);
  const size_t off = (size_t)k * 2 * c->Vh * site_bytes(dtype);
  const char* ep = (const char*)eta + off;
  for (int p = 0; p < 2; ++p) CK(dl::pack(B1, nn->act, p, p ? X.o[0]->ref() : X.e[0]->ref(), ep, dtype, c->st));
  if (s) {
    const char* sp = (const char*)s + off;
    CK(dl::pack(B1, P32, 0, se->ref(), sp, dtype, c->st));
    CK(dl::pack(B1, P32, 1, so->ref(), sp, dtype, c->st));
  }
  return DL_OK;
}

// 1 / |s_k|^2 for the n targets (host values)
dl_status target_norms(dl_nn* nn, int n, const void* s, int dtype, std::vector<double>& inv) {
  dl_ctx* c = nn->c;
  const Batch B1 = make_batch(c, 1);
  Field *se, *so;
  dl_status st;
  if ((st = ensure_field(c, "nn_se", P32, B1, &se)) || (st = ensure_field(c, "nn_so", P32, B1, &so))) return st;
  std::vector<double> h(2 * (size_t)n);
  double* dn;
  void* p;
  if ((st = ensure_buf(c, "nn_norms", sizeof(double) * 2 * std::max(n, 1), &p)) != DL_OK) return st;
  dn = (double*)p;
  for (int k = 0; k < n; ++k) {
    const char* sp = (const char*)s + (size_t)k * 2 * c->Vh * site_bytes(dtype);
    CK(dl::pack(B1, P32, 0, se->ref(), sp, dtype, c->st));
    CK(dl::pack(B1, P32, 1, so->ref(), sp, dtype, c->st));
    CK(dl::pdot(B1, P32, se->ref(), so->ref(), se->ref(), so->ref(), c->partial, dn + 2 * k, c->st));
  }
  CK(cudaMemcpyAsync(h.data(), dn, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  inv.resize(n);
  for (int k = 0; k < n; ++k) {
    if (!(h[2 * k] > 0.0)) return fail(c, DL_ERR_ARG, "a training target is zero");
    inv[k] = 1.0 / h[2 * k];
  }
  return DL_OK;
}

// Forward, loss and backward of the pairs idx[0..n) with inverse target norms
// inv_dev (device, per listed pair); weight-gradient partials accumulate in
// nn->wpart.  Returns the summed loss of the pairs.  kind 0: |N eta - s|^2 / |s|^2;
// kind 1 (residual, s unused, inv = 1 / |eta|^2): |M_u N eta - eta|^2 / |eta|^2, whose
// output gradient M_u^+ (M_u y - eta) / |eta|^2 is formed in FP32 with the stencil.
dl_status loss_grad_pairs(dl_nn* nn, const void* eta, const void* s, int dtype, const int* idx, int n,
                          const double* inv_dev, const std::vector<double>& inv_host, double* loss, int kind = 0) {
  dl_ctx* c = nn->c;
  dl_status st;
  Acts X, G;
  if ((st = get_acts(nn, "x", 0, X)) || (st = get_acts(nn, "g", 1, G))) return st;
  const Batch B1 = make_batch(c, 1);
  Field *se, *so;
  if ((st = ensure_field(c, "nn_se", P32, B1, &se)) || (st = ensure_field(c, "nn_so", P32, B1, &so))) return st;
  if (2 * n > nn->nloss) {
    if (nn->dscal) cudaFree(nn->dscal);
    nn->dscal = nullptr;
    nn->nloss = 0;
    CK(cudaMalloc((void**)&nn->dscal, sizeof(double) * (2 + 2 * (size_t)n)));
    nn->nloss = 2 * n;
  }
  double* lossd = nn->dscal + 2;
  Field *ye = nullptr, *yo = nullptr, *me = nullptr, *mo = nullptr, *ze = nullptr, *zo = nullptr;
  if (kind == 1) {
    if ((st = ensure_field(c, "nn_ye", P32, B1, &ye)) || (st = ensure_field(c, "nn_yo", P32, B1, &yo)) ||
        (st = ensure_field(c, "nn_me", P32, B1, &me)) || (st = ensure_field(c, "nn_mo", P32, B1, &mo)) ||
        (st = ensure_field(c, "nn_ze", nn->act, B1, &ze)) || (st = ensure_field(c, "nn_zo", nn->act, B1, &zo)))
      return st;
    CK(dl::zero(B1, nn->act, ze->ref(), nullptr, c->st));
    CK(dl::zero(B1, nn->act, zo->ref(), nullptr, c->st));
  }
  GaugeSet g{c->g64, c->g32, c->g16};
  const EpiSet Em = epiB(B1, CK_MK, 0, 0, 1, 1);    // out_p = R_u in_p - kappa D in_{1-p}: M_u
  const EpiSet Ed = epiB(B1, CK_MK, 0, 0, 1, -1);   // M_u^+ (dagger projectors)
  for (int q = 0; q < n; ++q) {
    if ((st = pack_pair(nn, eta, kind == 1 ? eta : s, dtype, idx[q], X, se, so)) != DL_OK) return st;
    if ((st = forward(nn, X)) != DL_OK) return st;
    if (kind == 0) {
      for (int p = 0; p < 2; ++p) {
        CK(dl::nn_lossgrad(B1, nn->act, p ? X.o[nn->nl]->ref() : X.e[nn->nl]->ref(), p ? so->ref() : se->ref(),
                           p ? G.o[nn->nl]->ref() : G.e[nn->nl]->ref(), inv_dev + q, c->partial, c->st));
        CK(dl::sum_partials(B1, c->partial, lossd + 2 * q + p, 0, 0, 1, c->st));
      }
    } else {
      // y in FP32; m = eta - M_u y (|m|^2 is the loss); then G = (0 - M_u^+ m) / |eta|^2
      CK(dl::copy(B1, P32, nn->act, ye->ref(), X.e[nn->nl]->ref(), nullptr, c->st));
      CK(dl::copy(B1, P32, nn->act, yo->ref(), X.o[nn->nl]->ref(), nullptr, c->st));
      CK(dl::dslash(B1, P32, c->rec32, EPI_AUX, false, 0, yo->ref(), ye->ref(), me->ref(), g, Em, nullptr, nullptr, NOF,
                    NOF, NOF, nullptr, c->st));
      CK(dl::dslash(B1, P32, c->rec32, EPI_AUX, false, 1, ye->ref(), yo->ref(), mo->ref(), g, Em, nullptr, nullptr, NOF,
                    NOF, NOF, nullptr, c->st));
      CK(dl::xmy_norm(B1, P32, me->ref(), se->ref(), me->ref(), nullptr, c->partial, c->st));
      CK(dl::sum_partials(B1, c->partial, lossd + 2 * q, 0, 0, 1, c->st));
      CK(dl::xmy_norm(B1, P32, mo->ref(), so->ref(), mo->ref(), nullptr, c->partial, c->st));
      CK(dl::sum_partials(B1, c->partial, lossd + 2 * q + 1, 0, 0, 1, c->st));
      CK(dl::dslash(B1, P32, c->rec32, EPI_AUX, true, 0, mo->ref(), me->ref(), ye->ref(), g, Ed, nullptr, nullptr, NOF,
                    NOF, NOF, nullptr, c->st));
      CK(dl::dslash(B1, P32, c->rec32, EPI_AUX, true, 1, me->ref(), mo->ref(), yo->ref(), g, Ed, nullptr, nullptr, NOF,
                    NOF, NOF, nullptr, c->st));
      CK(dl::nn_lossgrad(B1, nn->act, ze->ref(), ye->ref(), G.e[nn->nl]->ref(), inv_dev + q, c->partial, c->st));
      CK(dl::nn_lossgrad(B1, nn->act, zo->ref(), yo->ref(), G.o[nn->nl]->ref(), inv_dev + q, c->partial, c->st));
    }
    if ((st = backward(nn, X, G)) != DL_OK) return st;
  }
  std::vector<double> h(2 * (size_t)n);
  CK(cudaMemcpyAsync(h.data(), lossd, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  double tot = 0.0;
  for (int q = 0; q < n; ++q) tot += (h[2 * q] + h[2 * q + 1]) * inv_host[q];
  *loss = tot;
  return DL_OK;
}

bool valid_nn(const dl_nn* nn) { return nn && nn->c && nn->W; }

}  // namespace

// Learned map for the truncated solver method: x = N(eta) column by column of a
// block (fields in precision P32, B single-lattice with the block's columns).
namespace dlh {
dl_status nn_map_block(dl_nn* nn, dl_ctx* c, const Batch& B, Field* ee, Field* eo, Field* xe, Field* xo) {
  if (!valid_nn(nn) || nn->c != c) return fail(c, DL_ERR_ARG, "lp_net belongs to another context");
  if (ee->prec != P32 || xe->prec != P32) return fail(c, DL_ERR_ARG, "learned LP map needs FP32 fields");
  dl_status st;
  Acts X;
  if ((st = get_acts(nn, "x", 0, X)) != DL_OK) return st;
  const LatDesc& L = B.lat[0];
  const int lg = L.lognpad;
  for (int j = 0; j < L.ncol; ++j) {
    CK(dl::copy_col(L, nn->act, P32, X.e[0]->ref(), 0, 0, ee->ref(), lg, j, c->st));
    CK(dl::copy_col(L, nn->act, P32, X.o[0]->ref(), 0, 0, eo->ref(), lg, j, c->st));
    if ((st = forward(nn, X)) != DL_OK) return st;
    CK(dl::copy_col(L, P32, nn->act, xe->ref(), lg, j, X.e[nn->nl]->ref(), 0, 0, c->st));
    CK(dl::copy_col(L, P32, nn->act, xo->ref(), lg, j, X.o[nn->nl]->ref(), 0, 0, c->st));
  }
  return check_tc(nn);
}
}  // namespace dlh

extern "C" {

dl_status dl_nn_create(dl_ctx* c, int n_layers, int channels, int act_prec, dl_nn** out) try {
  dl_status s;
  if (!out) return DL_ERR_ARG;
  *out = nullptr;
  if ((s = check_ctx(c, true)) != DL_OK) return s;
  if (n_layers < 1 || n_layers > NN_MAX_LAYERS || channels < 1 || channels > 16 ||
      !(act_prec == DL_F32 || act_prec == DL_BF16))
    return fail(c, DL_ERR_ARG, "dl_nn_create: 1..16 layers, 1..16 channels, DL_F32 or DL_BF16 activations");
  if (!(c->rec32 == 12 || c->rec32 == 8)) return fail(c, DL_ERR_ARG, "dl_nn_create: FP32 links must use recon 12 or 8");
  dl_nn* nn = new dl_nn();
  nn->c = c;
  nn->nl = n_layers;
  nn->C = channels;
  nn->act = act_prec == DL_F32 ? P32 : PBF;
  int sms = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev);
  nn->slots = std::max(1, sms);
  // layer l's weight-gradient partials: slots consecutive copies of its 36 C_out C_in weights
  for (int l = 0; l < n_layers; ++l) {
    nn->ci.push_back(l == 0 ? 1 : channels);
    nn->co.push_back(l == n_layers - 1 ? 1 : channels);
    nn->woff.push_back(nn->nw);
    nn->poff.push_back(nn->npart * nn->slots);
    nn->nw += (size_t)36 * nn->co[l] * nn->ci[l];
    nn->npart += (size_t)36 * nn->co[l] * nn->ci[l];
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&nn->W, sizeof(float2) * nn->nw);
  if (e == cudaSuccess) e = cudaMalloc((void**)&nn->grad, sizeof(float2) * nn->nw);
  if (e == cudaSuccess) e = cudaMalloc((void**)&nn->m, sizeof(float2) * nn->nw);
  if (e == cudaSuccess) e = cudaMalloc((void**)&nn->v, sizeof(float2) * nn->nw);
  if (e == cudaSuccess) e = cudaMalloc((void**)&nn->wpart, sizeof(float2) * nn->npart * nn->slots);
  if (e == cudaSuccess) e = cudaMalloc((void**)&nn->dscal, sizeof(double) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&nn->tcB, TC_LAYER_BYTES * n_layers);
  if (e == cudaSuccess) e = cudaMalloc(&nn->tcBa, TC_LAYER_BYTES * n_layers);
  if (e == cudaSuccess) e = cudaMalloc((void**)&nn->Wa, sizeof(float2) * 36 * 16 * 16);
  if (e == cudaSuccess) e = cudaMalloc((void**)&nn->tc_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(nn->tc_err, 0, sizeof(int));
  nn->use_tc = nn->act == PBF;  // bfloat16 activations run on the tensor cores by default
  if (e == cudaSuccess) {
    nn->nloss = 2;
    e = cudaMemset(nn->W, 0, sizeof(float2) * nn->nw);
  }
  if (e == cudaSuccess) e = cudaMemset(nn->m, 0, sizeof(float2) * nn->nw);
  if (e == cudaSuccess) e = cudaMemset(nn->v, 0, sizeof(float2) * nn->nw);
  if (e != cudaSuccess) {
    dl_nn_destroy(nn);
    return cuda_fail(c, e, "dl_nn_create: device allocation");
  }
  *out = nn;
  return DL_OK;
} DL_CATCH(c)

void dl_nn_destroy(dl_nn* nn) try {
  if (!nn) return;
  if (nn->c) {
    cudaSetDevice(nn->c->dev);
    cudaStreamSynchronize(nn->c->st);
  }
  cudaFree(nn->W);
  cudaFree(nn->grad);
  cudaFree(nn->m);
  cudaFree(nn->v);
  cudaFree(nn->wpart);
  cudaFree(nn->dscal);
  cudaFree(nn->tcB);
  cudaFree(nn->tcBa);
  cudaFree(nn->Wa);
  cudaFree(nn->tc_err);
  delete nn;
} catch (...) {
}

long long dl_nn_weight_count(const dl_nn* nn) { return nn ? (long long)nn->nw : 0; }

dl_status dl_nn_set_tensor_cores(dl_nn* nn, int enable) try {
  if (!valid_nn(nn)) return DL_ERR_ARG;
  if (enable && nn->act != PBF) return fail(nn->c, DL_ERR_ARG, "the tensor-core forward needs bfloat16 activations");
  nn->use_tc = enable != 0;
  nn->tc_dirty = true;
  return DL_OK;
} DL_CATCH((nn ? nn->c : nullptr))

dl_status dl_nn_set_weights(dl_nn* nn, const float* w) try {
  if (!valid_nn(nn) || !w) return DL_ERR_ARG;
  dl_ctx* c = nn->c;
  dl_status s;
  if ((s = enter(c)) != DL_OK) return s;
  CK(cudaMemcpyAsync(nn->W, w, sizeof(float2) * nn->nw, cudaMemcpyHostToDevice, c->st));
  nn->tc_dirty = true;
  CK(cudaMemsetAsync(nn->m, 0, sizeof(float2) * nn->nw, c->st));
  CK(cudaMemsetAsync(nn->v, 0, sizeof(float2) * nn->nw, c->st));
  CK(cudaStreamSynchronize(c->st));
  nn->adam_t = 0;
  return leave(c);
} DL_CATCH((nn ? nn->c : nullptr))

dl_status dl_nn_get_weights(dl_nn* nn, float* w) try {
  if (!valid_nn(nn) || !w) return DL_ERR_ARG;
  dl_ctx* c = nn->c;
  dl_status s;
  if ((s = enter(c)) != DL_OK) return s;
  CK(cudaMemcpyAsync(w, nn->W, sizeof(float2) * nn->nw, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  return leave(c);
} DL_CATCH((nn ? nn->c : nullptr))

dl_status dl_nn_apply(dl_nn* nn, int n, const void* in, void* out, int dtype) try {
  if (!valid_nn(nn)) return DL_ERR_ARG;
  dl_ctx* c = nn->c;
  if (!in || !out || n < 1 || (dtype != DL_C128 && dtype != DL_C64)) return fail(c, DL_ERR_ARG, "dl_nn_apply: bad argument");
  dl_status s;
  if ((s = enter(c)) != DL_OK) return s;
  Acts X;
  if ((s = get_acts(nn, "x", 0, X)) != DL_OK) return s;
  const Batch B1 = make_batch(c, 1);
  for (int k = 0; k < n; ++k) {
    const size_t off = (size_t)k * 2 * c->Vh * site_bytes(dtype);
    for (int p = 0; p < 2; ++p) CK(dl::pack(B1, nn->act, p, p ? X.o[0]->ref() : X.e[0]->ref(), (const char*)in + off, dtype, c->st));
    if ((s = forward(nn, X)) != DL_OK) return s;
    for (int p = 0; p < 2; ++p)
      CK(dl::unpack(B1, nn->act, p, (char*)out + off, p ? X.o[nn->nl]->ref() : X.e[nn->nl]->ref(), dtype, c->st));
  }
  if ((s = check_tc(nn)) != DL_OK) return s;
  return leave(c);
} DL_CATCH((nn ? nn->c : nullptr))

dl_status dl_nn_apply_adjoint(dl_nn* nn, int n, const void* in, void* out, int dtype) try {
  if (!valid_nn(nn)) return DL_ERR_ARG;
  dl_ctx* c = nn->c;
  if (!in || !out || n < 1 || (dtype != DL_C128 && dtype != DL_C64))
    return fail(c, DL_ERR_ARG, "dl_nn_apply_adjoint: bad argument");
  dl_status s;
  if ((s = enter(c)) != DL_OK) return s;
  Acts G;
  if ((s = get_acts(nn, "g", 0, G)) != DL_OK) return s;
  const Batch B1 = make_batch(c, 1);
  for (int k = 0; k < n; ++k) {
    const size_t off = (size_t)k * 2 * c->Vh * site_bytes(dtype);
    for (int p = 0; p < 2; ++p)
      CK(dl::pack(B1, nn->act, p, p ? G.o[nn->nl]->ref() : G.e[nn->nl]->ref(), (const char*)in + off, dtype, c->st));
    if ((s = adjoint(nn, G)) != DL_OK) return s;
    for (int p = 0; p < 2; ++p)
      CK(dl::unpack(B1, nn->act, p, (char*)out + off, p ? G.o[0]->ref() : G.e[0]->ref(), dtype, c->st));
  }
  return leave(c);
} DL_CATCH((nn ? nn->c : nullptr))

dl_status dl_nn_loss_grad(dl_nn* nn, int n, const void* eta, const void* s, int dtype, double* loss, float* grad) try {
  if (!valid_nn(nn)) return DL_ERR_ARG;
  dl_ctx* c = nn->c;
  if (!eta || !s || n < 1 || (dtype != DL_C128 && dtype != DL_C64)) return fail(c, DL_ERR_ARG, "dl_nn_loss_grad: bad argument");
  dl_status st;
  if ((st = enter(c)) != DL_OK) return st;
  std::vector<double> inv;
  if ((st = target_norms(nn, n, s, dtype, inv)) != DL_OK) return st;
  void* p;
  if ((st = ensure_buf(c, "nn_inv", sizeof(double) * n, &p)) != DL_OK) return st;
  double* inv_dev = (double*)p;
  CK(cudaMemcpyAsync(inv_dev, inv.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->st));
  std::vector<int> idx(n);
  for (int k = 0; k < n; ++k) idx[k] = k;
  if ((st = zero_wpart(nn)) != DL_OK) return st;
  double L = 0.0;
  if ((st = loss_grad_pairs(nn, eta, s, dtype, idx.data(), n, inv_dev, inv, &L)) != DL_OK) return st;
  if ((st = reduce_grad(nn)) != DL_OK) return st;
  if (grad) CK(cudaMemcpyAsync(grad, nn->grad, sizeof(float2) * nn->nw, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (loss) *loss = L;
  if ((st = check_tc(nn)) != DL_OK) return st;
  return leave(c);
} DL_CATCH((nn ? nn->c : nullptr))

dl_status dl_nn_loss_grad_residual(dl_nn* nn, int n, const void* eta, int dtype, double* loss, float* grad) try {
  if (!valid_nn(nn)) return DL_ERR_ARG;
  dl_ctx* c = nn->c;
  if (!eta || n < 1 || (dtype != DL_C128 && dtype != DL_C64))
    return fail(c, DL_ERR_ARG, "dl_nn_loss_grad_residual: bad argument");
  dl_status st;
  if ((st = enter(c)) != DL_OK) return st;
  std::vector<double> inv;
  if ((st = target_norms(nn, n, eta, dtype, inv)) != DL_OK) return st;
  void* p;
  if ((st = ensure_buf(c, "nn_inv", sizeof(double) * n, &p)) != DL_OK) return st;
  double* inv_dev = (double*)p;
  CK(cudaMemcpyAsync(inv_dev, inv.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->st));
  std::vector<int> idx(n);
  for (int k = 0; k < n; ++k) idx[k] = k;
  if ((st = zero_wpart(nn)) != DL_OK) return st;
  double L = 0.0;
  if ((st = loss_grad_pairs(nn, eta, nullptr, dtype, idx.data(), n, inv_dev, inv, &L, 1)) != DL_OK) return st;
  if ((st = reduce_grad(nn)) != DL_OK) return st;
  if (grad) CK(cudaMemcpyAsync(grad, nn->grad, sizeof(float2) * nn->nw, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (loss) *loss = L;
  if ((st = check_tc(nn)) != DL_OK) return st;
  return leave(c);
} DL_CATCH((nn ? nn->c : nullptr))

dl_status dl_nn_train(dl_nn* nn, const dl_nn_train_params* prm, int n_pairs, const void* eta, const void* s, int dtype,
                      double* loss_hist) try {
  if (!valid_nn(nn)) return DL_ERR_ARG;
  dl_ctx* c = nn->c;
  if (!prm || !eta || n_pairs < 1 || prm->steps < 0 || prm->batch < 1 || prm->batch > n_pairs ||
      !(prm->lr > 0.0) || !(prm->beta1 >= 0.0 && prm->beta1 < 1.0) || !(prm->beta2 >= 0.0 && prm->beta2 < 1.0) ||
      !(prm->eps > 0.0) || (dtype != DL_C128 && dtype != DL_C64) || (prm->loss != 0 && prm->loss != 1) ||
      (prm->loss == 0 && !s))
    return fail(c, DL_ERR_ARG, "dl_nn_train: bad parameters");
  dl_status st;
  if ((st = enter(c)) != DL_OK) return st;
  std::vector<double> inv;
  // 1 / |s|^2 for the solution loss, 1 / |eta|^2 for the residual loss
  if ((st = target_norms(nn, n_pairs, prm->loss == 1 ? eta : s, dtype, inv)) != DL_OK) return st;
  void* p;
  if ((st = ensure_buf(c, "nn_inv", sizeof(double) * n_pairs, &p)) != DL_OK) return st;
  double* inv_all = (double*)p;
  CK(cudaMemcpyAsync(inv_all, inv.data(), sizeof(double) * n_pairs, cudaMemcpyHostToDevice, c->st));
  if ((st = ensure_buf(c, "nn_invb", sizeof(double) * prm->batch, &p)) != DL_OK) return st;
  double* inv_b = (double*)p;
  // seeded Fisher-Yates order per pass over the pairs (splitmix64 stream)
  uint64_t state = prm->seed;
  auto next = [&]() {
    state += 0x9E3779B97F4A7C15ULL;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  };
  std::vector<int> order(n_pairs);
  int pos = n_pairs;
  std::vector<int> idx(prm->batch);
  std::vector<double> invh(prm->batch);
  for (int step = 0; step < prm->steps; ++step) {
    for (int q = 0; q < prm->batch; ++q) {
      if (pos == n_pairs) {
        for (int k = 0; k < n_pairs; ++k) order[k] = k;
        for (int k = n_pairs - 1; k > 0; --k) std::swap(order[k], order[next() % (uint64_t)(k + 1)]);
        pos = 0;
      }
      idx[q] = order[pos++];
      invh[q] = inv[idx[q]];
      CK(cudaMemcpyAsync(inv_b + q, inv_all + idx[q], sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    }
    if ((st = zero_wpart(nn)) != DL_OK) return st;
    double L = 0.0;
    if ((st = loss_grad_pairs(nn, eta, s, dtype, idx.data(), prm->batch, inv_b, invh, &L, prm->loss)) != DL_OK) return st;
    if ((st = reduce_grad(nn)) != DL_OK) return st;
    nn->adam_t += 1;
    CK(dl::nn_adam(nn->W, nn->grad, nn->m, nn->v, nn->nw, (float)prm->lr, (float)prm->beta1, (float)prm->beta2,
                   (float)prm->eps, nn->adam_t, 1.f / (float)prm->batch, c->st));
    nn->tc_dirty = true;
    if (loss_hist) loss_hist[step] = L / prm->batch;
  }
  CK(cudaStreamSynchronize(c->st));
  if ((st = check_tc(nn)) != DL_OK) return st;
  return leave(c);
} DL_CATCH((nn ? nn->c : nullptr))

dl_status dl_fgcr_solve(dl_ctx* c, dl_nn* nn, const dl_fgcr_params* prm, int n, const void* src, void* sol, int dtype,
                        dl_fgcr_stats* stats) try {
  dl_status s;
  if ((s = check_ctx(c, true)) != DL_OK) return s;
  if (!prm || !src || !sol || n < 1 || n > DL_MAX_RHS || !(prm->tol > 0.0) || prm->max_iter < 1 || prm->restart < 1 ||
      prm->restart > 256 || !(prm->inner_tol > 0.0 && prm->inner_tol < 1.0) || (prm->flavour != 1 && prm->flavour != -1) ||
      (dtype != DL_C128 && dtype != DL_C64))
    return fail(c, DL_ERR_ARG, "dl_fgcr_solve: bad parameters");
  if (nn && (!valid_nn(nn) || nn->c != c)) return fail(c, DL_ERR_ARG, "dl_fgcr_solve: network of another context");
  if ((s = enter(c)) != DL_OK) return s;
  auto t0 = std::chrono::steady_clock::now();
  const Batch B1 = make_batch(c, 1);
  if ((s = ensure_partial(c, B1)) != DL_OK) return s;
  const int m = prm->restart;
  Field *be, *bo, *xe, *xo, *re, *ro, *te, *to, *r3e, *r3o, *e3e, *e3o;
  if ((s = ensure_field(c, "fg_be", P64, B1, &be)) || (s = ensure_field(c, "fg_bo", P64, B1, &bo)) ||
      (s = ensure_field(c, "fg_xe", P64, B1, &xe)) || (s = ensure_field(c, "fg_xo", P64, B1, &xo)) ||
      (s = ensure_field(c, "fg_re", P64, B1, &re)) || (s = ensure_field(c, "fg_ro", P64, B1, &ro)) ||
      (s = ensure_field(c, "fg_te", P64, B1, &te)) || (s = ensure_field(c, "fg_to", P64, B1, &to)) ||
      (s = ensure_field(c, "fg_r3e", P32, B1, &r3e)) || (s = ensure_field(c, "fg_r3o", P32, B1, &r3o)) ||
      (s = ensure_field(c, "fg_e3e", P32, B1, &e3e)) || (s = ensure_field(c, "fg_e3o", P32, B1, &e3o)))
    return s;
  std::vector<Field*> ze(m), zo(m), we(m), wo(m);
  for (int j = 0; j < m; ++j) {
    const std::string k = std::to_string(j);
    if ((s = ensure_field(c, "fg_ze" + k, P32, B1, &ze[j])) || (s = ensure_field(c, "fg_zo" + k, P32, B1, &zo[j])) ||
        (s = ensure_field(c, "fg_we" + k, P32, B1, &we[j])) || (s = ensure_field(c, "fg_wo" + k, P32, B1, &wo[j])))
      return s;
  }
  const bool normal = prm->normal != 0;
  Field *u3e, *u3o, *v3e, *v3o;  // normal mode: normalised true residual, and M z before M^+
  if ((s = ensure_field(c, "fg_u3e", P32, B1, &u3e)) || (s = ensure_field(c, "fg_u3o", P32, B1, &u3o)) ||
      (s = ensure_field(c, "fg_v3e", P32, B1, &v3e)) || (s = ensure_field(c, "fg_v3o", P32, B1, &v3o)))
    return s;
  Acts X, G;
  if (nn && (s = get_acts(nn, "x", 0, X)) != DL_OK) return s;
  if (nn && normal && (s = get_acts(nn, "g", 0, G)) != DL_OK) return s;
  void* p;
  if ((s = ensure_buf(c, "fg_scal", sizeof(double) * 2, &p)) != DL_OK) return s;
  double* dsc = (double*)p;
  GaugeSet g{c->g64, c->g32, c->g16};
  const EpiSet E = epiB(B1, CK_MK, 0, 0, 1, prm->flavour);    // out_p = R_f in_p - kappa D in_{1-p}
  const EpiSet Ed = epiB(B1, CK_MK, 0, 0, 1, -prm->flavour);  // the same for M^+ (dagger projectors, -mu)
  long long nop = 0, nnn = 0;
  auto applyMd = [&](int prec, bool dag, Field* ie, Field* io, Field* oe, Field* oo) -> dl_status {
    const int gr = grec_of(c, prec);
    const EpiSet& EE = dag ? Ed : E;
    CK(dl::dslash(B1, prec, gr, EPI_AUX, dag, 0, io->ref(), ie->ref(), oe->ref(), g, EE, nullptr, nullptr, NOF, NOF, NOF,
                  nullptr, c->st));
    CK(dl::dslash(B1, prec, gr, EPI_AUX, dag, 1, ie->ref(), io->ref(), oo->ref(), g, EE, nullptr, nullptr, NOF, NOF, NOF,
                  nullptr, c->st));
    ++nop;
    return DL_OK;
  };
  auto applyM = [&](int prec, Field* ie, Field* io, Field* oe, Field* oo) -> dl_status {
    return applyMd(prec, false, ie, io, oe, oo);
  };
  // the inner operator: M, or M^+ M in normal mode
  auto applyA = [&](Field* ie, Field* io, Field* oe, Field* oo) -> dl_status {
    if (!normal) return applyM(P32, ie, io, oe, oo);
    dl_status s2 = applyMd(P32, false, ie, io, v3e, v3o);
    if (s2 != DL_OK) return s2;
    return applyMd(P32, true, v3e, v3o, oe, oo);
  };
  auto dot = [&](int prec, Field* ae, Field* ao, Field* b2e, Field* b2o, double& dr, double& di) -> dl_status {
    CK(dl::pdot(B1, prec, ae->ref(), ao->ref(), b2e->ref(), b2o->ref(), c->partial, dsc, c->st));
    double h[2];
    CK(cudaMemcpyAsync(h, dsc, sizeof(h), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    dr = h[0];
    di = h[1];
    return DL_OK;
  };
  auto axpy = [&](int prec, double ar, double ai, Field* x1e, Field* x1o, Field* ye, Field* yo) -> dl_status {
    CK(dl::caxpy(B1, prec, ar, ai, x1e->ref(), ye->ref(), c->st));
    CK(dl::caxpy(B1, prec, ar, ai, x1o->ref(), yo->ref(), c->st));
    return DL_OK;
  };
  auto precond = [&](Field* ie, Field* io, Field* oe, Field* oo) -> dl_status {
    if (!nn) {
      CK(dl::copy(B1, P32, P32, oe->ref(), ie->ref(), nullptr, c->st));
      CK(dl::copy(B1, P32, P32, oo->ref(), io->ref(), nullptr, c->st));
      return DL_OK;
    }
    if (normal) {  // P = N N^+ (symmetric positive definite for an invertible N)
      CK(dl::copy(B1, nn->act, P32, G.e[nn->nl]->ref(), ie->ref(), nullptr, c->st));
      CK(dl::copy(B1, nn->act, P32, G.o[nn->nl]->ref(), io->ref(), nullptr, c->st));
      dl_status s3 = adjoint(nn, G);
      if (s3 != DL_OK) return s3;
      CK(dl::copy(B1, nn->act, nn->act, X.e[0]->ref(), G.e[0]->ref(), nullptr, c->st));
      CK(dl::copy(B1, nn->act, nn->act, X.o[0]->ref(), G.o[0]->ref(), nullptr, c->st));
    } else {
      CK(dl::copy(B1, nn->act, P32, X.e[0]->ref(), ie->ref(), nullptr, c->st));
      CK(dl::copy(B1, nn->act, P32, X.o[0]->ref(), io->ref(), nullptr, c->st));
    }
    dl_status s2 = forward(nn, X);
    if (s2 != DL_OK) return s2;
    CK(dl::copy(B1, P32, nn->act, oe->ref(), X.e[nn->nl]->ref(), nullptr, c->st));
    CK(dl::copy(B1, P32, nn->act, oo->ref(), X.o[nn->nl]->ref(), nullptr, c->st));
    ++nnn;
    return DL_OK;
  };
  dl_fgcr_stats st;
  memset(&st, 0, sizeof(st));
  bool any_nc = false;
  double dr, di;
  for (int k = 0; k < n; ++k) {
    const size_t off = (size_t)k * 2 * c->Vh * site_bytes(dtype);
    CK(dl::pack(B1, P64, 0, be->ref(), (const char*)src + off, dtype, c->st));
    CK(dl::pack(B1, P64, 1, bo->ref(), (const char*)src + off, dtype, c->st));
    if ((s = dot(P64, be, bo, be, bo, dr, di)) != DL_OK) return s;
    const double bn = std::sqrt(dr);
    CK(dl::zero(B1, P64, xe->ref(), nullptr, c->st));
    CK(dl::zero(B1, P64, xo->ref(), nullptr, c->st));
    CK(dl::copy(B1, P64, P64, re->ref(), be->ref(), nullptr, c->st));
    CK(dl::copy(B1, P64, P64, ro->ref(), bo->ref(), nullptr, c->st));
    int iters = 0, cycles = 0;
    double rn = bn;
    while (bn > 0.0 && rn > prm->tol * bn && iters < prm->max_iter) {
      ++cycles;
      // inner FP32 cycle on the normalised residual (normal mode: on M^+ of it)
      Field* ue = normal ? u3e : r3e;
      Field* uo = normal ? u3o : r3o;
      CK(dl::copy(B1, P32, P64, ue->ref(), re->ref(), nullptr, c->st));
      CK(dl::copy(B1, P32, P64, uo->ref(), ro->ref(), nullptr, c->st));
      if ((s = axpy(P32, 1.0 / rn - 1.0, 0.0, ue, uo, ue, uo)) != DL_OK) return s;
      double rho0 = 1.0;
      if (normal) {
        if ((s = applyMd(P32, true, u3e, u3o, r3e, r3o)) != DL_OK) return s;
        if ((s = dot(P32, r3e, r3o, r3e, r3o, dr, di)) != DL_OK) return s;
        rho0 = std::sqrt(std::max(dr, 0.0));
      }
      CK(dl::zero(B1, P32, e3e->ref(), nullptr, c->st));
      CK(dl::zero(B1, P32, e3o->ref(), nullptr, c->st));
      for (int j = 0; j < m && iters < prm->max_iter; ++j) {
        if ((s = precond(r3e, r3o, ze[j], zo[j])) != DL_OK) return s;
        if ((s = applyA(ze[j], zo[j], we[j], wo[j])) != DL_OK) return s;
        for (int i = 0; i < j; ++i) {  // modified Gram-Schmidt against the unit directions w_i
          if ((s = dot(P32, we[i], wo[i], we[j], wo[j], dr, di)) != DL_OK) return s;
          if ((s = axpy(P32, -dr, -di, we[i], wo[i], we[j], wo[j])) != DL_OK) return s;
          if ((s = axpy(P32, -dr, -di, ze[i], zo[i], ze[j], zo[j])) != DL_OK) return s;
        }
        if ((s = dot(P32, we[j], wo[j], we[j], wo[j], dr, di)) != DL_OK) return s;
        const double nu = std::sqrt(dr);
        if (!(nu > 0.0) || !std::isfinite(nu)) break;
        if ((s = axpy(P32, 1.0 / nu - 1.0, 0.0, we[j], wo[j], we[j], wo[j])) != DL_OK) return s;
        if ((s = axpy(P32, 1.0 / nu - 1.0, 0.0, ze[j], zo[j], ze[j], zo[j])) != DL_OK) return s;
        double ar, ai;
        if ((s = dot(P32, we[j], wo[j], r3e, r3o, ar, ai)) != DL_OK) return s;
        if ((s = axpy(P32, ar, ai, ze[j], zo[j], e3e, e3o)) != DL_OK) return s;
        if ((s = axpy(P32, -ar, -ai, we[j], wo[j], r3e, r3o)) != DL_OK) return s;
        ++iters;
        if ((s = dot(P32, r3e, r3o, r3e, r3o, dr, di)) != DL_OK) return s;
        const double rho = std::sqrt(std::max(dr, 0.0));
        if (rho <= prm->inner_tol * rho0 || (!normal && rho * rn <= 0.5 * prm->tol * bn)) break;
      }
      // x += |r| e; r = b - M x in FP64
      CK(dl::copy(B1, P64, P32, te->ref(), e3e->ref(), nullptr, c->st));
      CK(dl::copy(B1, P64, P32, to->ref(), e3o->ref(), nullptr, c->st));
      if ((s = axpy(P64, rn, 0.0, te, to, xe, xo)) != DL_OK) return s;
      if ((s = applyM(P64, xe, xo, te, to)) != DL_OK) return s;
      CK(dl::xmy_norm(B1, P64, re->ref(), be->ref(), te->ref(), nullptr, c->partial, c->st));
      CK(dl::xmy_norm(B1, P64, ro->ref(), bo->ref(), to->ref(), nullptr, c->partial, c->st));
      if ((s = dot(P64, re, ro, re, ro, dr, di)) != DL_OK) return s;
      rn = std::sqrt(std::max(dr, 0.0));
    }
    if (bn > 0.0 && rn > prm->tol * bn) any_nc = true;
    CK(dl::unpack(B1, P64, 0, (char*)sol + off, xe->ref(), dtype, c->st));
    CK(dl::unpack(B1, P64, 1, (char*)sol + off, xo->ref(), dtype, c->st));
    st.iters[k] = iters;
    st.cycles[k] = cycles;
    st.true_resid[k] = bn > 0.0 ? rn / bn : 0.0;
  }
  CK(cudaStreamSynchronize(c->st));
  if (nn && (s = check_tc(nn)) != DL_OK) return s;
  st.op_applications = nop;
  st.nn_applications = nnn;
  st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = st;
  if ((s = leave(c)) != DL_OK) return s;
  return any_nc ? fail(c, DL_NOT_CONVERGED, "dl_fgcr_solve: max_iter reached") : DL_OK;
} DL_CATCH(c)

}  // extern "C"
