// Internal entry points of the step/rounding orchestration (see step.cu, prim.cu).
#pragma once
#include "common.cuh"
#include "small.cuh"

namespace ttk {
// S: storage type of the cores; T: arithmetic of the passes over the merged core (TSQR leaves
// and merges, update pass).  Small cores, norms, rank decisions and energies are FP64.
template <typename S, typename T>
tt_status round_impl(tt_context* ctx, tt_tensor* x, double tol, int rmax, Bump& ws);
template <typename S, typename T>
tt_status step_impl(tt_context* ctx, const tt_plan* p, tt_tensor* I, double tol, int rmax, double* energy,
                    Bump& ws);
template <typename S>
tt_status energy_density_impl(tt_context* ctx, const tt_plan* p, const tt_tensor* x, double* out, Bump& ws);
template <typename S>
tt_status apply_transport_impl(tt_context* ctx, const tt_plan* p, const tt_tensor* in, tt_tensor* out);
template <typename S>
tt_status axpy_impl(tt_context* ctx, double alpha, const tt_tensor* x, tt_tensor* y);
template <typename S>
tt_status dot_into(cudaStream_t s, const tt_tensor* x, const tt_tensor* y, double* out, double* scratch,
                   size_t cap);
template <typename S>
tt_status internal_ranks_impl(tt_context* ctx, const tt_plan* p, const tt_tensor* x, double delta, int* ranks,
                              double* sig_nu, long nsig_nu, double* sig_x, long nsig_x, Bump& ws);
template <typename S>
tt_status dot_impl(tt_context* ctx, const tt_tensor* x, const tt_tensor* y, double* out, Bump& ws);
}  // namespace ttk
