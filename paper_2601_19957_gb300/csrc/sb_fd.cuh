// sb_fd.cuh -- launch interface of the black-box central-difference derivatives (App. A.4)
// and the uniform-correlation probe (Sec. 3.7.2).
#pragma once
#include "sb_internal.cuh"

namespace sb {

// Perturbed points of one call: 4d + 3, plus 2 d (d - 1) with the full Hessian.
int64_t fd_rows(int d, bool full);
// Points evaluated per batch.
int fd_chunk_rows(int d);
// Doubles of scratch (l at every row, one chunk of points, its |z|^2 partials).
size_t fd_scratch_elems(int d, int K, bool full);
// grad (may be null), hdiag, H (full only), b (may be null) at x; pv needs a_k.
void launch_fd(const ProbView &pv, const double *x, double eps_g, double eps_h, bool full, double *scratch,
               double *grad, double *hdiag, double *H, double *b, cudaStream_t s);

}  // namespace sb
