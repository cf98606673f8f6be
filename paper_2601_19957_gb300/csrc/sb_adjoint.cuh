// sb_adjoint.cuh -- FP64 adjoint of log Z (adjoint.cu).
#pragma once
#include <vector>

#include "sb_internal.cuh"
#include "sb_laplace.cuh"

namespace sb {

constexpr int kMaxAdjModes = 1024;

struct AdjWs {
    double *P, *H, *M, *Z, *R, *qpart, *gbar, *ell, *GK, *V, *T, *cvec, *eps, *gam, *u, *trWP, *pi;
    double *PY, *y;  // P_k (W gbar - W g_k) per component [K][d]; a d-vector
    int32_t *info, *one, *onehot;
    uint32_t *bar;  // grid-barrier state of the cooperative factorisation
};

void adjoint_carve(Carver &cv, AdjWs &w, int d, int K);
sb_status adjoint_run(const ProbView &pv, const AdjWs &w, const double *modes, const double *logZk, int n_modes,
                      double grad_logZ, double *dmu, double *dL, cudaStream_t s);

}  // namespace sb
