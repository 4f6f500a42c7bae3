// Launchers shared between the discloop translation units (host side).
#pragma once

#include "dl_internal.cuh"

// Per-column CG scalars, struct of arrays: S[slot * DL_NCMAX + gc]
#define DL_NCMAX 256
#define DL_NS 8
#define DL_S_RR 0
#define DL_S_RR0 1
#define DL_S_ALPHA 2
#define DL_S_BETA 3
#define DL_S_PAP 4
#define DL_S_MAXR 5
#define DL_S_RRNEW 6
#define DL_S_TMP 7

#define DL_FLAG_CONVERGED 1
#define DL_FLAG_BREAKDOWN 2
#define DL_FLAG_UPDATE 4

namespace dl {
// blas
cudaError_t copy(const Batch& B, int pd, int ps, FieldRef dst, FieldRef src, const int* mask, cudaStream_t st);
cudaError_t accum(const Batch& B, int ph, int pl, FieldRef x, FieldRef y, const int* mask, int zero_y, cudaStream_t st);
cudaError_t xmy_norm(const Batch& B, int prec, FieldRef r, FieldRef b, FieldRef a, const int* mask, double* partial,
                     cudaStream_t st);
// out (po) = a (pa) - b (pb), evaluated in a's arithmetic (FP32 out from a high-precision a and an FP32 b)
cudaError_t diff(const Batch& B, int po, int pa, int pb, FieldRef out, FieldRef a, FieldRef b, cudaStream_t st);
cudaError_t norm2(const Batch& B, int prec, FieldRef v, const int* mask, double* partial, cudaStream_t st);
cudaError_t xpay(const Batch& B, int prec, FieldRef p, FieldRef r, const double* beta, const int* mask, cudaStream_t st);
cudaError_t twist(const Batch& B, int prec, FieldRef out, FieldRef in, const EpiSet& ep, const int* mask, cudaStream_t st);
cudaError_t zero(const Batch& B, int prec, FieldRef v, const int* mask, cudaStream_t st);
cudaError_t sum_partials(const Batch& B, const double* partial, double* out, int stride, int slot, int ncols_total,
                         cudaStream_t st);
cudaError_t cg_alpha(int ncols, double* S, int* active, int* flags, cudaStream_t st);
cudaError_t cg_beta(int ncols, double* S, int* active, int* flags, int* iters, double tol2, double delta, cudaStream_t st);
// Loop condition of the CG graph: sets h, or writes *cont when cont != nullptr (plain launches)
cudaError_t cg_cond(int ncols, const int* active, const int* flags, int* counter, const int* limit, int* wait,
                    cudaGraphConditionalHandle h, int* cont, cudaStream_t st);

// layout (single-lattice batches)
cudaError_t pack(const Batch& B, int prec, int parity, FieldRef dst, const void* natural, int dtype, cudaStream_t st);
cudaError_t unpack(const Batch& B, int prec, int parity, void* natural, FieldRef src, int dtype, cudaStream_t st);
// S (optional): only the sites of these time slices get noise, the rest zero
cudaError_t noise_z4(const Batch& B, int prec, int parity, FieldRef dst, unsigned long long seed,
                     unsigned long long first, int quadrant, cudaStream_t st, Slices S = Slices{0, 1, 0});
cudaError_t pack_gauge(const LatDesc& L, const double* links_dev, void* g64, void* gdf, void* g32, int rec32, void* g16,
                       int rec16, cudaStream_t st);

// contractions
cudaError_t contract_sites(const Batch& B, int prec, int mode, int with_deriv, FieldRef s_e, FieldRef s_o, FieldRef eta_e,
                           FieldRef eta_o, const void* g64, double2* W, cudaStream_t st);
cudaError_t dft_pass(const double2* in, double2* out, long long nb, int len, long long stride, int m, double2* phase,
                     int fp32, cudaStream_t st);
// G1 (and the DFT passes' buffers) hold float pairs for P32, double-float pairs for PDF
// and double pairs for P64; dft_pass / contract_finalize take the kind as fp32 = 1 / 2 / 0
// S: the time slices covered (all_slices(T), or the slices of a time-diluted source;
// G1 .. G3 then hold only those slices, finalize writes zeros on the others)
cudaError_t contract_x(const Batch& B, int prec, int mode, int with_deriv, FieldRef s_e, FieldRef s_o, FieldRef eta_e,
                       FieldRef eta_o, const void* g64, const void* g32, int rec32, int mx, double2* phx, double2* G1,
                       Slices S, cudaStream_t st);
cudaError_t contract_finalize(const Batch& B, int with_deriv, int np, const int* mom_dev, int mx, int my, int mz,
                              const double2* G3, int fp32, double pre_re, double pre_im, double2* out, int accumulate,
                              Slices S, cudaStream_t st);
cudaError_t hpe_exact(double kappa, double amu, int flavour, double2* out16, cudaStream_t st);
cudaError_t add_exact_p0(const Batch& B, int np, int nd, int ip0, const double2* exact16, double scale, double2* out,
                         Slices S, cudaStream_t st);
cudaError_t col_accumulate(const double2* blk, const double2* sub, int ncol, long long per_col, double sign, double2* acc,
                           cudaStream_t st);
cudaError_t observables(const double2* l1, const double2* l2, int ncol, int T, int np, int nd, int ip0, double* obs,
                        cudaStream_t st);
cudaError_t combine(const double2* x, const double2* y, double a, double b, long long n, double2* out, cudaStream_t st);
// learned preconditioner (dl_network.cu)
cudaError_t nn_forward(const LatDesc& L, int prec, int grec, int parity, FieldRef xe, FieldRef xo, FieldRef y,
                       const void* g32, const float2* W, int ci, int co, int lgin, int lgout, cudaStream_t st);
cudaError_t nn_backward_x(const LatDesc& L, int prec, int grec, int parity, FieldRef ge, FieldRef go, FieldRef gx,
                          const void* g32, const float2* W, int ci, int co, int lgin, int lgout, cudaStream_t st);
cudaError_t nn_backward_w(const LatDesc& L, int prec, int grec, int parity, FieldRef xe, FieldRef xo, FieldRef gp,
                          const void* g32, int ci, int co, int lgin, int lgout, float2* partial, int slots,
                          cudaStream_t st);
// the same weight-gradient partials on the tensor cores (bfloat16 activations; `slots` persistent
// CTAs, at most one per 32-site tile); err is set when a bounded wait ran out
cudaError_t nn_backward_w_tc(const LatDesc& L, int grec, int parity, FieldRef xe, FieldRef xo, FieldRef gp,
                             const void* g32, int ci, int co, int lgin, int lgout, float2* partial, int slots, int* err,
                             cudaStream_t st);
cudaError_t nn_wsum(const float2* partial, int nslice, size_t nW, float2* grad, cudaStream_t st);
// tensor-core forward (bfloat16 activations): B chunks of a layer (36 x 2 KB), then the layer
cudaError_t nn_tc_prep(const float2* W, int ci, int co, void* Bc, cudaStream_t st);
// weights of the adjoint layer (C_out -> C_in channels, [9][4][ci][co]): with them the
// forward kernels compute the input gradient
cudaError_t nn_adj_weights(const float2* W, int ci, int co, float2* Wa, cudaStream_t st);
cudaError_t nn_forward_tc(const LatDesc& L, int grec, int parity, FieldRef xe, FieldRef xo, FieldRef y, const void* g32,
                          const void* Bc, int ci, int co, int lgin, int lgout, int* err, cudaStream_t st);
cudaError_t nn_lossgrad(const Batch& B, int prec, FieldRef y, FieldRef s, FieldRef g, const double* inv_ns, double* partial,
                        cudaStream_t st);
cudaError_t nn_adam(float2* W, const float2* grad, float2* m, float2* v, size_t n, float lr, float b1, float b2, float eps,
                    int step, float gscale, cudaStream_t st);
// <a, b> over both parities of a single-column field, written to out[0] (re), out[1] (im) on the device
cudaError_t pdot(const Batch& B, int prec, FieldRef ae, FieldRef ao, FieldRef be, FieldRef bo, double* partial,
                 double* out, cudaStream_t st);
cudaError_t copy_col(const LatDesc& L, int pd, int ps, FieldRef dst, int lgd, int cd, FieldRef src, int lgs, int cs,
                     cudaStream_t st);
// y += alpha x (single column, complex alpha)
cudaError_t caxpy(const Batch& B, int prec, double ar, double ai, FieldRef x, FieldRef y, cudaStream_t st);
}  // namespace dl
