// fd.cu -- black-box derivatives of l by central differences (App. A.4) and
// the uniform-correlation probe (Sec. 3.7.2), FP64.
//
// l is used as a black box: every derivative comes from l at perturbed points,
// evaluated in chunks by the batched likelihood (one batch per chunk of rows).
// Row layout of one call (R rows in all):
//   0                      x
//   1 + 2i, 2 + 2i         x + eps_g e_i, x - eps_g e_i          (gradient)
//   1 + 2d + 2i, 2 + 2d+2i x + eps_h e_i, x - eps_h e_i          (Hessian diagonal)
//   1 + 4d, 2 + 4d         x + eps_h v, x - eps_h v, v = 1/sqrt(d) (probe)
//   3 + 4d + 4p + {0..3}   x +- eps_h e_i +- eps_h e_j, pair p = (i < j) in
//                          row-major order, signs ++, +-, -+, --  (off-diagonal)
// and then
//   grad_i = (l(x + eps_g e_i) - l(x - eps_g e_i)) / (2 eps_g)
//   H_ii   = (l(x + eps_h e_i) - 2 l(x) + l(x - eps_h e_i)) / eps_h^2
//   H_ij   = (l_++ - l_+- - l_-+ + l_--) / (4 eps_h^2), mirrored
//   b      = (v^T H v - mean H_ii) / (d - 1), v^T H v from the second difference along v.
// The Hessians are of l itself (negative definite at a maximum).
#include "sb_fd.cuh"

namespace sb {

namespace {

__host__ __device__ inline int64_t fd_pair_start(int64_t i, int64_t d) { return i * d - i * (i + 1) / 2; }

// pair index p -> (i, j), i < j, row-major over the strict upper triangle
__device__ void fd_pair(int64_t p, int d, int &i, int &j) {
    const double dd = (double)d;
    int64_t ii = (int64_t)floor((2.0 * dd - 1.0 - sqrt((2.0 * dd - 1.0) * (2.0 * dd - 1.0) - 8.0 * (double)p)) / 2.0);
    if (ii < 0) ii = 0;
    if (ii > d - 2) ii = d - 2;
    while (ii > 0 && fd_pair_start(ii, d) > p) --ii;
    while (ii < d - 2 && fd_pair_start(ii + 1, d) <= p) ++ii;
    i = (int)ii;
    j = (int)(p - fd_pair_start(ii, d) + ii + 1);
}

// warp per row of the chunk [r0, r0 + nr): the perturbed point
__global__ void __launch_bounds__(256) k_fd_points(int64_t r0, int nr, int d, const double *x, double eps_g,
                                                   double eps_h, double *P) {
    const int lane = threadIdx.x & 31;
    const int w = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (w >= nr) return;
    const int64_t row = r0 + w;
    double *p = P + (size_t)w * d;
    int i = -1, j = -1;
    double ai = 0.0, aj = 0.0;
    bool probe = false;
    if (row == 0) {
    } else if (row <= 2 * (int64_t)d) {
        i = (int)((row - 1) / 2);
        ai = ((row - 1) % 2) ? -eps_g : eps_g;
    } else if (row <= 4 * (int64_t)d) {
        i = (int)((row - 1 - 2 * d) / 2);
        ai = ((row - 1 - 2 * d) % 2) ? -eps_h : eps_h;
    } else if (row <= 4 * (int64_t)d + 2) {
        probe = true;
        ai = row == 4 * (int64_t)d + 1 ? eps_h : -eps_h;
    } else {
        const int64_t q = row - (4 * (int64_t)d + 3);
        fd_pair(q / 4, d, i, j);
        const int sg = (int)(q % 4);
        ai = sg < 2 ? eps_h : -eps_h;
        aj = (sg % 2) == 0 ? eps_h : -eps_h;
    }
    if (probe) {
        const double step = mul_rn(ai, div_rn(1.0, sqrt((double)d)));
        for (int c = lane; c < d; c += 32) p[c] = add_rn(x[c], step);
        return;
    }
    for (int c = lane; c < d; c += 32) {
        double v = x[c];
        if (c == i) v = add_rn(v, ai);
        if (c == j) v = add_rn(v, aj);
        p[c] = v;
    }
}

__global__ void __launch_bounds__(256) k_fd_axes(int d, const double *f, double eps_g, double eps_h, double *grad,
                                                 double *hdiag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d) return;
    const double f0 = f[0];
    if (grad) grad[i] = div_rn(sub_rn(f[1 + 2 * i], f[2 + 2 * i]), mul_rn(2.0, eps_g));
    const double fp = f[1 + 2 * d + 2 * i], fm = f[2 + 2 * d + 2 * i];
    hdiag[i] = div_rn(add_rn(sub_rn(fp, mul_rn(2.0, f0)), fm), mul_rn(eps_h, eps_h));
}

__global__ void __launch_bounds__(256) k_fd_pairs(int d, const double *f, double eps_h, double *H) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t np = (int64_t)d * (d - 1) / 2;
    if (p >= np) return;
    int i, j;
    fd_pair(p, d, i, j);
    const double *q = f + 4 * (int64_t)d + 3 + 4 * p;
    const double h = div_rn(add_rn(sub_rn(sub_rn(q[0], q[1]), q[2]), q[3]), mul_rn(mul_rn(4.0, eps_h), eps_h));
    H[(size_t)i * d + j] = h;
    H[(size_t)j * d + i] = h;
}

__global__ void __launch_bounds__(32) k_fd_finish(int d, const double *f, double eps_h, const double *hdiag, double *H,
                                                  double *b) {
    if (threadIdx.x != 0) return;
    if (H)
        for (int i = 0; i < d; ++i) H[(size_t)i * d + i] = hdiag[i];
    if (b) {
        if (d < 2) {
            *b = 0.0;
            return;
        }
        const double f0 = f[0], fp = f[1 + 4 * d], fm = f[2 + 4 * d];
        const double vhv = div_rn(add_rn(sub_rn(fp, mul_rn(2.0, f0)), fm), mul_rn(eps_h, eps_h));
        double a = 0.0;
        for (int i = 0; i < d; ++i) a = add_rn(a, hdiag[i]);
        a = div_rn(a, (double)d);
        *b = div_rn(sub_rn(vhv, a), (double)(d - 1));
    }
}

}  // namespace

int64_t fd_rows(int d, bool full) { return 4 * (int64_t)d + 3 + (full ? 2 * (int64_t)d * (d - 1) : 0); }

int fd_chunk_rows(int d) {
    int64_t c = ((int64_t)32 << 20) / d;  // 256 MB of points per chunk
    if (c < 64) c = 64;
    if (c > (1 << 20)) c = 1 << 20;
    return (int)c;
}

size_t fd_scratch_elems(int d, int K, bool full) {
    const int c = fd_chunk_rows(d);
    return (size_t)fd_rows(d, full) + (size_t)c * d + lik_f64_qpart_elems(d, K, c);
}

void launch_fd(const ProbView &pv, const double *x, double eps_g, double eps_h, bool full, double *scratch,
               double *grad, double *hdiag, double *H, double *b, cudaStream_t s) {
    const int d = pv.d, K = pv.K;
    const int64_t R = fd_rows(d, full);
    const int C = fd_chunk_rows(d);
    double *f = scratch;
    double *P = f + R;
    double *qpart = P + (size_t)C * d;
    for (int64_t r0 = 0; r0 < R; r0 += C) {
        const int nr = (int)(R - r0 < C ? R - r0 : C);
        note_launch();
        k_fd_points<<<(unsigned)(((int64_t)nr * 32 + 255) / 256), 256, 0, s>>>(r0, nr, d, x, eps_g, eps_h, P);
        LikF64Args a{};
        a.d = d;
        a.K = K;
        a.mu = pv.mu;
        a.L = pv.L;
        a.a = pv.a;
        a.c = pv.c;
        a.X = P;
        a.n_rows = nr;
        a.qpart = qpart;
        a.ell = f + r0;
        a.ell_sign = 1.0;
        a.out_by_walker = 0;
        launch_lik_f64_points(a, false, s);
    }
    note_launch();
    k_fd_axes<<<(d + 255) / 256, 256, 0, s>>>(d, f, eps_g, eps_h, grad, hdiag);
    if (full && d > 1) {
        const int64_t np = (int64_t)d * (d - 1) / 2;
        note_launch();
        k_fd_pairs<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(d, f, eps_h, H);
    }
    note_launch();
    k_fd_finish<<<1, 32, 0, s>>>(d, f, eps_h, hdiag, full ? H : nullptr, b);
}

}  // namespace sb
