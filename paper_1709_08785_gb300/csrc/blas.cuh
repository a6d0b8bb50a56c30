// Launchers of the fused BLAS-1 kernels (blas.cu).  n is the number of
// sites processed (Vh_pad for a half vector, 2*Vh_pad for a full one).
#pragma once

#include "ctx.cuh"

namespace qcd {

size_t hvec_elems(const Geom &g, int prec);
int state_init(qcd_ctx *c, SolverState *st, double tol2, double tol2_rel, int maxit, double bd_eps, int unit);
int set_tol2(qcd_ctx *c, SolverState *dst, const SolverState *src, int slot, double factor);
int state_mark_done(qcd_ctx *c, SolverState *st);
int blas_update_s(qcd_ctx *c, int prec, int n, HVec r, HVec q, SolverState *st);
int blas_update_x(qcd_ctx *c, int prec, int n, HVec x, HVec p, HVec r, HVec t, HVec rt, SolverState *st);
int blas_update_p(qcd_ctx *c, int prec, int n, HVec p, HVec r, HVec q, SolverState *st, int fin);
int blas_finish_half(qcd_ctx *c, int prec, int n, HVec x, HVec p, SolverState *st);
int blas_flex1(qcd_ctx *c, int prec, int n, HVec x, HVec v, HVec r, HVec q, SolverState *st);
int blas_flex2(qcd_ctx *c, int prec, int n, HVec x, HVec v, HVec r, HVec t, HVec rt, SolverState *st);
int blas_init(qcd_ctx *c, int prec, int n, HVec src, HVec r, HVec rt, HVec p, HVec x, int zero_x, SolverState *st,
              int fin);
int blas_norm2(qcd_ctx *c, int prec, int n, HVec a, SolverState *st, int fin);
int blas_dot(qcd_ctx *c, int prec, int n, HVec a, HVec b, SolverState *st, int fin, const int *done);
int blas_omega(qcd_ctx *c, int prec, int n, HVec t, HVec r, SolverState *st, const int *done);
int blas_inner_init(qcd_ctx *c, int ps, int pd, int n, HVec src, const double *src_norm2, HVec r, HVec rt, HVec p,
                    HVec x, const int *done);
int blas_lift(qcd_ctx *c, int ps, int pd, int n, HVec x, HVec v, const double *src_norm2, const int *done);

}  // namespace qcd
