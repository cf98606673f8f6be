// rays.cu -- sunburst ray directions and start selection (Sec. 3.5.1-3.5.2, Sec. 4.1).
//
// Directions: ray r, coordinate pair p draws one Philox4x32-10 block with
// counter (p, r, 'RAYS', 0) and key (seed lo, seed hi); its two 64-bit words
// give two uniforms, Box-Muller gives two standard normals, and the vector is
// scaled to unit length (uniform on S^{d-1}). t_exit,r = min_i half_i / |u_ri|
// is the distance from the box centre to the box surface along u_r.
//
// Start selection takes the n_starts smallest keys (tier, rank, -l, flat):
// tier 0 marks a discrete local maximum of l along its ray (the sign change of
// the ray derivative, Sec. 4.1), rank is the position of l inside its ray.
// The cut is found exactly: a histogram over (tier, rank) buckets picks the
// bucket holding the n_starts-th key, then a 12-pass 8-bit radix select over
// the 96-bit key (order-preserving bits of -l, flat index) inside that bucket.
// Selected samples are emitted in ascending flat index by an ordered scan.
#include "sb_internal.cuh"

namespace sb {

namespace {

__global__ void __launch_bounds__(256) k_ray_dirs(int d, int n_rays, uint32_t k0, uint32_t k1, const double *half,
                                                  double *u, double *texit) {
    const int lane = threadIdx.x & 31;
    const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= n_rays) return;
    double *ur = u + (size_t)r * d;
    const int npairs = (d + 1) / 2;
    double ss = 0.0;
    for (int p = lane; p < npairs; p += 32) {
        uint32_t c[4] = {(uint32_t)p, (uint32_t)r, 0x52415953u, 0u};
        philox4x32_10(c, k0, k1);
        const double u1 = unit_from_words(c[0], c[1]);
        const double u2 = unit_from_words(c[2], c[3]);
        const double rad = sqrt(-2.0 * log(u1));
        const double th = mul_rn(SB_TWO_PI, u2);
        const double x0 = mul_rn(rad, cos(th));
        ur[2 * p] = x0;
        ss += x0 * x0;
        if (2 * p + 1 < d) {
            const double x1 = mul_rn(rad, sin(th));
            ur[2 * p + 1] = x1;
            ss += x1 * x1;
        }
    }
    const double nrm = sqrt(warp_sum(ss));
    __syncwarp();
    for (int i = lane; i < d; i += 32) ur[i] = div_rn(ur[i], nrm);
    __syncwarp();
    const double tmin = warp_exit_min(lane, d, ur, half);
    if (lane == 0) texit[r] = tmin;
}

// The same rays for the mixed-precision path, generated in FP32 (the tensor-core
// operands carry fewer bits): the same Philox counters, uniforms from the top 24 bits
// of each 64-bit pair, Box-Muller with FP32 transcendentals, normalised in FP32 and
// widened to FP64; t_exit in FP64 for the widened direction, so the last sample of a
// ray lies on the box surface.
__global__ void __launch_bounds__(256) k_ray_dirs_f32(int d, int n_rays, uint32_t k0, uint32_t k1, const double *half,
                                                      double *u, double *texit) {
    const int lane = threadIdx.x & 31;
    const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= n_rays) return;
    double *ur = u + (size_t)r * d;
    const int npairs = (d + 1) / 2;
    constexpr int kPer = 16;  // pairs a lane keeps in registers before the norm is known
    float x[2 * kPer];
    float ss = 0.f;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const int p = lane + 32 * q;
        x[2 * q] = x[2 * q + 1] = 0.f;
        if (p < npairs) {
            uint32_t c[4] = {(uint32_t)p, (uint32_t)r, 0x52415953u, 0u};
            philox4x32_10(c, k0, k1);
            const float u1 = ((float)(c[0] >> 8) + 0.5f) * (1.0f / 16777216.0f);
            const float u2 = ((float)(c[2] >> 8) + 0.5f) * (1.0f / 16777216.0f);
            const float rad = sqrtf(-2.0f * logf(u1));
            float sn, cs;
            sincospif(2.0f * u2, &sn, &cs);
            x[2 * q] = rad * cs;
            x[2 * q + 1] = 2 * p + 1 < d ? rad * sn : 0.f;
            ss += x[2 * q] * x[2 * q] + x[2 * q + 1] * x[2 * q + 1];
        }
    }
    // pairs beyond the register block (d > 1024) are stored unnormalised first
    for (int p = lane + 32 * kPer; p < npairs; p += 32) {
        uint32_t c[4] = {(uint32_t)p, (uint32_t)r, 0x52415953u, 0u};
        philox4x32_10(c, k0, k1);
        const float u1 = ((float)(c[0] >> 8) + 0.5f) * (1.0f / 16777216.0f);
        const float u2 = ((float)(c[2] >> 8) + 0.5f) * (1.0f / 16777216.0f);
        const float rad = sqrtf(-2.0f * logf(u1));
        float sn, cs;
        sincospif(2.0f * u2, &sn, &cs);
        const float x0 = rad * cs;
        ur[2 * p] = x0;
        ss += x0 * x0;
        if (2 * p + 1 < d) {
            const float x1 = rad * sn;
            ur[2 * p + 1] = x1;
            ss += x1 * x1;
        }
    }
    const float inv = 1.0f / sqrtf(warp_sum(ss));
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const int p = lane + 32 * q;
        if (p < npairs) {
            ur[2 * p] = (double)(x[2 * q] * inv);
            if (2 * p + 1 < d) ur[2 * p + 1] = (double)(x[2 * q + 1] * inv);
        }
    }
    for (int p = lane + 32 * kPer; p < npairs; p += 32) {
        ur[2 * p] = (double)((float)ur[2 * p] * inv);
        if (2 * p + 1 < d) ur[2 * p + 1] = (double)((float)ur[2 * p + 1] * inv);
    }
    __syncwarp();
    const double tmin = warp_exit_min(lane, d, ur, half);
    if (lane == 0) texit[r] = tmin;
}

// One warp per ray: tier and rank of every sample, histogram of buckets.
__global__ void __launch_bounds__(128) k_ray_bucket(const double *ell, int n_rays, int S, int32_t *bucket,
                                                    uint32_t *hist) {
    extern __shared__ double sh[];  // [4][S]
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int r = blockIdx.x * 4 + wl;
    double *row = sh + (size_t)wl * S;
    if (r < n_rays)
        for (int j = lane; j < S; j += 32) row[j] = ell[(size_t)r * S + j];
    __syncwarp();
    if (r >= n_rays) return;
    for (int j = lane; j < S; j += 32) {
        const double l = row[j];
        const double left = j > 0 ? row[j - 1] : -INFINITY;
        const double right = j + 1 < S ? row[j + 1] : -INFINITY;
        const int tier = (l > left && l >= right) ? 0 : 1;
        int rank = 0;
        for (int j2 = 0; j2 < S; ++j2) {
            const double l2 = row[j2];
            rank += (l2 > l || (l2 == l && j2 < j)) ? 1 : 0;
        }
        const int b = tier * S + rank;
        bucket[(size_t)r * S + j] = b;
        atomicAdd(&hist[b], 1u);
    }
}

// state: [0] cut bucket, [1] need (1-based rank inside the bucket), [2] key hi prefix, [3] key lo prefix
__global__ void k_pick_bucket(uint32_t *hist, int nbins, int n_starts, uint64_t *state) {
    if (threadIdx.x == 0) {
        uint64_t cum = 0;
        int b = 0;
        for (; b < nbins; ++b) {
            if (cum + hist[b] >= (uint64_t)n_starts) break;
            cum += hist[b];
        }
        state[0] = (uint64_t)b;
        state[1] = (uint64_t)n_starts - cum;
        state[2] = 0;
        state[3] = 0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
}

__device__ __forceinline__ void sample_key(const double *ell, int64_t f, uint64_t &hi, uint32_t &lo) {
    hi = ~ordered_bits(ell[f]);  // ascending hi = descending l
    lo = (uint32_t)f;
}

// Digit histogram of pass p (0..11) over the 96-bit keys in the cut bucket.
__global__ void __launch_bounds__(256) k_digit_hist(const double *ell, const int32_t *bucket, int64_t total, int pass,
                                                    const uint64_t *state, uint32_t *hist) {
    __shared__ uint32_t sh[256];
    sh[threadIdx.x] = 0;
    __syncthreads();
    const int64_t cut = (int64_t)state[0];
    const uint64_t phi = state[2];
    const uint32_t plo = (uint32_t)state[3];
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < total; f += (int64_t)gridDim.x * blockDim.x) {
        if (bucket[f] != cut) continue;
        uint64_t hi;
        uint32_t lo;
        sample_key(ell, f, hi, lo);
        uint32_t digit;
        bool match;
        if (pass < 8) {
            const int sh_hi = 64 - 8 * pass;  // bits above the current digit
            match = pass == 0 ? true : ((hi >> sh_hi) == (phi >> sh_hi));
            digit = (uint32_t)((hi >> (56 - 8 * pass)) & 0xffu);
        } else {
            const int q = pass - 8;
            const int sh_lo = 32 - 8 * q;
            match = (hi == phi) && (q == 0 ? true : ((lo >> sh_lo) == (plo >> sh_lo)));
            digit = (lo >> (24 - 8 * q)) & 0xffu;
        }
        if (match) atomicAdd(&sh[digit], 1u);
    }
    __syncthreads();
    if (sh[threadIdx.x]) atomicAdd(&hist[threadIdx.x], sh[threadIdx.x]);
}

__global__ void k_digit_decide(uint32_t *hist, int pass, uint64_t *state) {
    if (threadIdx.x == 0) {
        uint64_t need = state[1], cum = 0;
        uint32_t dg = 0;
        for (; dg < 256; ++dg) {
            if (cum + hist[dg] >= need) break;
            cum += hist[dg];
        }
        state[1] = need - cum;
        if (pass < 8)
            state[2] |= (uint64_t)dg << (56 - 8 * pass);
        else
            state[3] |= (uint64_t)dg << (24 - 8 * (pass - 8));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
}

__device__ __forceinline__ bool is_selected(const double *ell, const int32_t *bucket, int64_t f,
                                            const uint64_t *state) {
    const int64_t b = bucket[f];
    const int64_t cut = (int64_t)state[0];
    if (b < cut) return true;
    if (b > cut) return false;
    uint64_t hi;
    uint32_t lo;
    sample_key(ell, f, hi, lo);
    const uint64_t khi = state[2];
    const uint32_t klo = (uint32_t)state[3];
    return hi < khi || (hi == khi && lo <= klo);
}

constexpr int SEL_BLOCK = 1024;

__global__ void __launch_bounds__(SEL_BLOCK) k_sel_count(const double *ell, const int32_t *bucket, int64_t total,
                                                         const uint64_t *state, int32_t *blockcnt) {
    const int64_t f = (int64_t)blockIdx.x * SEL_BLOCK + threadIdx.x;
    const int sel = (f < total) && is_selected(ell, bucket, f, state);
    const int cnt = __syncthreads_count(sel);
    if (threadIdx.x == 0) blockcnt[blockIdx.x] = cnt;
}

__global__ void __launch_bounds__(SEL_BLOCK) k_sel_scatter(const double *ell, const int32_t *bucket, int64_t total,
                                                           const uint64_t *state, const int32_t *blockcnt,
                                                           int64_t *idx) {
    __shared__ int warp_tot[32];
    __shared__ long long s_base;
    // offset of this block = sum of the preceding block counts
    long long part = 0;
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += SEL_BLOCK) part += blockcnt[b];
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) warp_tot[wid] = (int)part;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long s = 0;
        for (int w = 0; w < SEL_BLOCK / 32; ++w) s += warp_tot[w];
        s_base = s;
    }
    __syncthreads();
    const int64_t f = (int64_t)blockIdx.x * SEL_BLOCK + threadIdx.x;
    const int sel = (f < total) && is_selected(ell, bucket, f, state);
    const unsigned bal = __ballot_sync(0xffffffffu, sel);
    const int in_warp = __popc(bal & ((1u << lane) - 1u));
    __syncthreads();
    if (lane == 0) warp_tot[wid] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < SEL_BLOCK / 32; ++w) {
            const int t = warp_tot[w];
            warp_tot[w] = s;
            s += t;
        }
    }
    __syncthreads();
    if (sel) idx[s_base + warp_tot[wid] + in_warp] = f;
}

__global__ void __launch_bounds__(256) k_gather_starts(int d, const double *c, const double *u, const double *texit,
                                                       int n_steps, const int64_t *idx, const double *ell_all,
                                                       int n_starts, double *starts, double *ell_starts) {
    const int lane = threadIdx.x & 31;
    const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= n_starts) return;
    const int64_t f = idx[s];
    const int r = (int)(f / n_steps), j = (int)(f % n_steps);
    const double scale = mul_rn(div_rn((double)(j + 1), (double)n_steps), texit[r]);
    for (int i = lane; i < d; i += 32)
        starts[(size_t)s * d + i] = add_rn(c[i], mul_rn(scale, u[(size_t)r * d + i]));
    if (lane == 0) ell_starts[s] = ell_all[f];
}

}  // namespace

size_t select_blocks(int64_t total) { return (size_t)((total + SEL_BLOCK - 1) / SEL_BLOCK); }

void launch_ray_dirs(int d, int n_rays, uint64_t seed, const ProbView &pv, double *u, double *texit, bool fp32,
                     cudaStream_t s) {
    const int warps_per_block = 8;
    const unsigned grid = (unsigned)((n_rays + warps_per_block - 1) / warps_per_block);
    note_launch();
    if (fp32)
        k_ray_dirs_f32<<<grid, 256, 0, s>>>(d, n_rays, (uint32_t)seed, (uint32_t)(seed >> 32), pv.half, u, texit);
    else
        k_ray_dirs<<<grid, 256, 0, s>>>(d, n_rays, (uint32_t)seed, (uint32_t)(seed >> 32), pv.half, u, texit);
}

void launch_select_starts(const double *ell_all, int n_rays, int n_steps, int n_starts, const SelectWs &w,
                          cudaStream_t s) {
    const int64_t total = (int64_t)n_rays * n_steps;
    const int nbins = 2 * n_steps;
    cudaMemsetAsync(w.hist, 0, sizeof(uint32_t) * (size_t)(nbins > 256 ? nbins : 256), s);
    note_launch();
    k_ray_bucket<<<(n_rays + 3) / 4, 128, sizeof(double) * 4 * n_steps, s>>>(ell_all, n_rays, n_steps, w.bucket,
                                                                             w.hist);
    note_launch();
    k_pick_bucket<<<1, 256, 0, s>>>(w.hist, nbins, n_starts, w.state);
    const int hb = (int)((total + 255) / 256 < 1184 ? (total + 255) / 256 : 1184);
    for (int pass = 0; pass < 12; ++pass) {
        note_launch();
        k_digit_hist<<<hb, 256, 0, s>>>(ell_all, w.bucket, total, pass, w.state, w.hist);
        note_launch();
        k_digit_decide<<<1, 256, 0, s>>>(w.hist, pass, w.state);
    }
    const int nb = (int)select_blocks(total);
    note_launch();
    k_sel_count<<<nb, SEL_BLOCK, 0, s>>>(ell_all, w.bucket, total, w.state, w.blockcnt);
    note_launch();
    k_sel_scatter<<<nb, SEL_BLOCK, 0, s>>>(ell_all, w.bucket, total, w.state, w.blockcnt, w.idx);
}

void launch_gather_starts(const ProbView &pv, const double *u, const double *texit, int n_steps, const int64_t *idx,
                          const double *ell_all, int n_starts, double *starts, double *ell_starts, cudaStream_t s) {
    note_launch();
    k_gather_starts<<<(n_starts + 7) / 8, 256, 0, s>>>(pv.d, pv.c, u, texit, n_steps, idx, ell_all, n_starts, starts,
                                                       ell_starts);
}

}  // namespace sb
