// Gradient with respect to the kernel f (learnable kernels).
//
// out[u] = sum_v f(dhat(u, v)) F[v] is linear in the grid samples f_k, so for a
// loss L with g = dL/dout,
//     C[k] = dL/df_k = sum over ordered pairs (u, v) with dhat(u, v) = k of <g_u, F_v>,
// and dL/dtheta = sum_k (df(k delta)/dtheta) C[k]. The apply computes
// out = sum over calls (G - E) + leaf terms, so C decomposes the same way:
// per table job (a call's A-bins, or a component's b-bins, sign -1) the pair
// histogram of its bin sums,
//     H[k] = sum_{i, l} <gsum_i, fsum_l> [r_i + r_l + |x_i - x_l| = k],
// and per leaf the pair histogram of its vertices. H is a convolution along
// depth and a correlation along the backbone coordinate, so it is one 2D FFT
// correlation of the two bin tables per channel, summed over channels in the
// frequency domain (gsum in the real part and the coordinate-reversed fsum in
// the imaginary part of one complex transform per channel), then binned along
// j + |b| = k. All sums run in a fixed order: C is deterministic.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "kernels.cuh"

namespace tfi {
namespace grad {

using dev::cmul;
using dev::padded;
using dev::padded_size;

struct GradJob {
    int32_t kb, ke, lp1, lp2, maxr, maxx;
    int64_t hoff;   // offset of this job's histogram (length 2 maxr + maxx + 1)
};

__device__ __forceinline__ int brev_bits(int v, int bits) { return bits ? int(__brev(uint32_t(v)) >> (32 - bits)) : 0; }

// One CTA per job; shared memory: Z and ACC, padded_size(P1 P2) complex each.
__global__ void grad_fft_kernel(const GradJob *__restrict__ jobs, const int32_t *__restrict__ key_r,
                                const int32_t *__restrict__ key_x, int d, const float *__restrict__ gsum,
                                const float *__restrict__ fsum, const float2 *__restrict__ tw,
                                float *__restrict__ hist) {
    extern __shared__ float2 smz[];
    const GradJob jb = jobs[blockIdx.x];
    const int lp1 = jb.lp1, lp2 = jb.lp2, lnp = lp1 + lp2;
    const int NP = 1 << lnp, P1 = 1 << lp1, P2 = 1 << lp2;
    const int padnp = padded_size(NP);
    float2 *Z = smz, *ACC = smz + padnp;
    for (int i = threadIdx.x; i < padnp; i += blockDim.x) ACC[i] = make_float2(0.f, 0.f);
    const int nk = jb.ke - jb.kb;
    for (int c = 0; c < d; ++c) {
        for (int i = threadIdx.x; i < padnp; i += blockDim.x) Z[i] = make_float2(0.f, 0.f);
        __syncthreads();
        for (int t = threadIdx.x; t < nk; t += blockDim.x) {
            const int k = jb.kb + t, r = key_r[k], x = key_x[k];
            Z[padded(r * P2 + x)].x = gsum[int64_t(k) * d + c];
        }
        __syncthreads();
        for (int t = threadIdx.x; t < nk; t += blockDim.x) {
            const int k = jb.kb + t, r = key_r[k], x = key_x[k];
            Z[padded(r * P2 + ((P2 - x) & (P2 - 1)))].y = fsum[int64_t(k) * d + c];
        }
        __syncthreads();
        dev::fft_axis<false>(Z, padnp, 1, lp2, 1, lp1, P2, false, tw, false);
        dev::fft_axis<false>(Z, padnp, 1, lp1, P2, lp2, 1, true, tw, false);
        // acc += A^ B^ with A^ = (Z[f] + conj Z[-f]) / 2, B^ = (Z[f] - conj Z[-f]) / 2i
        for (int p = threadIdx.x; p < NP; p += blockDim.x) {
            const int p1 = p >> lp2, p2 = p & (P2 - 1);
            const int f1 = brev_bits(p1, lp1), f2 = brev_bits(p2, lp2);
            const int q = (brev_bits((P1 - f1) & (P1 - 1), lp1) << lp2) | brev_bits((P2 - f2) & (P2 - 1), lp2);
            const float2 z = Z[padded(p)], w = Z[padded(q)];
            const float2 z2 = cmul(z, z);
            const float2 wc = make_float2(w.x, -w.y);
            const float2 w2 = cmul(wc, wc);
            // (z^2 - conj(w)^2) / (4 i) = (im, -re) / 4
            const float re = z2.x - w2.x, im = z2.y - w2.y;
            ACC[padded(p)].x += 0.25f * im;
            ACC[padded(p)].y += -0.25f * re;
        }
        __syncthreads();
    }
    dev::fft_axis<true>(ACC, padnp, 1, lp1, P2, lp2, 1, true, tw, false);
    dev::fft_axis<true>(ACC, padnp, 1, lp2, 1, lp1, P2, false, tw, false);
    // H[j][b] = ACC / NP (real); bin j + min(b, P2 - b) = k
    const float inv = 1.f / float(NP);
    const int K = 2 * jb.maxr + jb.maxx + 1;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        float acc = 0.f;
        const int j0 = max(0, k - jb.maxx), j1 = min(k, 2 * jb.maxr);
        for (int j = j0; j <= j1; ++j) {
            const int b = k - j;
            acc += ACC[padded(j * P2 + (b & (P2 - 1)))].x;
            if (b > 0 && b < P2 - b) acc += ACC[padded(j * P2 + P2 - b)].x;
        }
        hist[jb.hoff + k] = acc * inv;
    }
}

template <typename T>
__device__ __forceinline__ float ldf(const T *p);
template <>
__device__ __forceinline__ float ldf<float>(const float *p) { return *p; }
template <>
__device__ __forceinline__ float ldf<__nv_bfloat16>(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

// Leaves, pass 1: for every ordered pair (i, j) of a leaf, its distance and
// <g_i, F_j>, at pair_off[leaf] + (i - lo) * s + (j - lo).
template <typename T>
__global__ void grad_leaf_pairs(const int32_t *__restrict__ leaf_ptr, const int64_t *__restrict__ pair_off,
                                const int32_t *__restrict__ leaf_vtx, const int32_t *__restrict__ leaf_dist,
                                const int32_t *__restrict__ leaf_pdist, const T *__restrict__ G,
                                const T *__restrict__ F, int d, float *__restrict__ pval, int32_t *__restrict__ pdst) {
    const int lf = blockIdx.x;
    const int lo = leaf_ptr[lf], hi = leaf_ptr[lf + 1], s = hi - lo;
    const int64_t base = pair_off[lf];
    for (int ii = threadIdx.x; ii < s; ii += blockDim.x) {
        const int i = lo + ii;
        const int64_t vi = leaf_vtx[i];
        const int di = leaf_dist[i];
        // self, then j = i+1 .. hi-1 (min over (i, j] grows), then j = i-1 .. lo (min over (j, i] grows)
        int m = 0x7fffffff;
        for (int step = 0; step < s; ++step) {
            int j, dist;
            if (step == 0) {
                j = i;
                dist = 0;
            } else if (i + step < hi) {
                j = i + step;
                m = min(m, leaf_pdist[j]);
                dist = di + leaf_dist[j] - 2 * m;
            } else {
                j = i - (step - (hi - 1 - i));
                if (j == i - 1) m = 0x7fffffff;
                m = min(m, leaf_pdist[j + 1]);
                dist = di + leaf_dist[j] - 2 * m;
            }
            const int64_t vj = leaf_vtx[j];
            float acc = 0.f;
            for (int c = 0; c < d; ++c) acc = fmaf(ldf<T>(G + vi * d + c), ldf<T>(F + vj * d + c), acc);
            pval[base + int64_t(ii) * s + (j - lo)] = acc;
            pdst[base + int64_t(ii) * s + (j - lo)] = dist;
        }
    }
}

// Leaves, pass 2: histogram of one leaf, one thread per distance, pairs in order.
__global__ void grad_leaf_hist(const int32_t *__restrict__ leaf_ptr, const int64_t *__restrict__ pair_off,
                               const int64_t *__restrict__ hist_off, const int32_t *__restrict__ hist_len,
                               const float *__restrict__ pval, const int32_t *__restrict__ pdst,
                               float *__restrict__ hist) {
    const int lf = blockIdx.x;
    const int s = leaf_ptr[lf + 1] - leaf_ptr[lf];
    const int64_t base = pair_off[lf];
    const int64_t np = int64_t(s) * s;
    for (int k = threadIdx.x; k < hist_len[lf]; k += blockDim.x) {
        float acc = 0.f;
        for (int64_t e = 0; e < np; ++e)
            if (pdst[base + e] == k) acc += pval[base + e];
        hist[hist_off[lf] + k] = acc;
    }
}

// C[k] = sum over segments (fixed order) of sign * hist_segment[k], in FP64.
__global__ void grad_reduce(int n_seg, const int64_t *__restrict__ seg_off, const int32_t *__restrict__ seg_len,
                            const float *__restrict__ seg_sign, const float *__restrict__ hist, int64_t len,
                            double *__restrict__ C) {
    for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < len; k += int64_t(gridDim.x) * blockDim.x) {
        double acc = 0.0;
        for (int sgm = 0; sgm < n_seg; ++sgm)
            if (k < seg_len[sgm]) acc += double(seg_sign[sgm]) * double(hist[seg_off[sgm] + k]);
        C[k] = acc;
    }
}

// dtheta[p] = sum_k (d f(k delta) / d theta_p) C[k], for the analytic kinds.
__global__ void grad_params(int kind, const double *__restrict__ params, int n_params, double delta,
                            const double *__restrict__ C, int64_t len, double *__restrict__ dtheta) {
    const int p = blockIdx.x;
    if (p >= n_params) return;
    __shared__ double part[256];
    double acc = 0.0;
    for (int64_t k = threadIdx.x; k < len; k += blockDim.x) {
        const double x = double(k) * delta;
        double df = 0.0;
        if (kind == 1) {  // expsum [a_i, b_i]
            const double a = params[p & ~1], b = params[p | 1];
            const double e = exp(-b * x);
            df = (p & 1) ? -a * x * e : e;
        } else if (kind == 2) {  // gauss [a, c]
            const double a = params[0], c = params[1], e = exp(-c * x * x);
            df = p == 0 ? e : -a * x * x * e;
        } else if (kind == 3) {  // rational [a, c, e, q]: a (1 + c x^e)^-q
            const double a = params[0], c = params[1], ee = params[2], q = params[3];
            const double xe = x > 0 ? pow(x, ee) : 0.0, base = 1.0 + c * xe;
            const double t = pow(base, -q);
            if (p == 0) df = t;
            else if (p == 1) df = -a * q * xe * t / base;
            else if (p == 2) df = x > 0 ? -a * q * c * xe * log(x) * t / base : 0.0;
            else df = -a * log(base) * t;
        } else if (kind == 4) {  // powexp [a, q, b]: a x^q exp(-b x)
            const double a = params[0], q = params[1], b = params[2];
            const double xq = x > 0 ? pow(x, q) : (q == 0 ? 1.0 : 0.0), e = exp(-b * x);
            if (p == 0) df = xq * e;
            else if (p == 1) df = x > 0 ? a * xq * log(x) * e : 0.0;
            else df = -a * x * xq * e;
        }
        acc += df * C[k];
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) part[threadIdx.x] += part[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) dtheta[p] = part[0];
}

}  // namespace grad
}  // namespace tfi
