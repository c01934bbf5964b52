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
#include "fft_x2.cuh"

namespace tfi {
namespace grad {

using dev::cmul;
using dev::padded;
using dev::padded_size;

struct GradJob {
    int32_t kb, ke, lp1, lp2, maxr, maxx;
    int64_t hoff;   // offset of this job's histograms: one per channel block, each 2 maxr + maxx + 1 long
    int32_t mode;   // 0: FFT correlation per channel block; 1: direct (pair dot products, then binning)
    int32_t pad;
    int64_t moff;   // direct jobs: offset of the nk x nk pair dot products
};

constexpr int kGradCB = 32;  // channels per CTA of grad_fft_kernel (blockIdx.y = channel block)

__device__ __forceinline__ int brev_bits(int v, int bits) { return bits ? int(__brev(uint32_t(v)) >> (32 - bits)) : 0; }

// One CTA per job and block of kGradCB channels; shared memory: Z and ACC,
// padded_size(P1 P2) complex each. Each channel block bins its own histogram
// (the transforms are linear, so the blocks' histograms add up to the job's).
__global__ void grad_fft_kernel(const GradJob *__restrict__ jobs, const int32_t *__restrict__ key_r,
                                const int32_t *__restrict__ key_x, int d, const float *__restrict__ gsum,
                                const float *__restrict__ fsum, const float2 *__restrict__ tw,
                                float *__restrict__ hist) {
    extern __shared__ float2 smz[];
    const GradJob jb = jobs[blockIdx.x];
    // direct jobs: grad_pair_dots / grad_direct_bin; one-dimensional FFT jobs: grad_fft1d_x2_kernel
    if (jb.mode != 0 || (jb.lp2 == 0 && jb.lp1 >= 1)) return;
    const int lp1 = jb.lp1, lp2 = jb.lp2, lnp = lp1 + lp2;
    const int NP = 1 << lnp, P1 = 1 << lp1, P2 = 1 << lp2;
    const int padnp = padded_size(NP);
    float2 *Z = smz, *ACC = smz + padnp;
    for (int i = threadIdx.x; i < padnp; i += blockDim.x) ACC[i] = make_float2(0.f, 0.f);
    const int nk = jb.ke - jb.kb;
    const int cb0 = blockIdx.y * kGradCB, cb1 = min(d, cb0 + kGradCB);
    for (int c = cb0; c < cb1; ++c) {
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
    __syncthreads();
    const float inv = 1.f / float(NP);
    const int K = 2 * jb.maxr + jb.maxx + 1;
    float *hblk = hist + int64_t(blockIdx.y) * K;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        float acc = 0.f;
        const int j0 = max(0, k - jb.maxx), j1 = min(k, 2 * jb.maxr);
        for (int j = j0; j <= j1; ++j) {
            const int b = k - j;
            acc += ACC[padded(j * P2 + (b & (P2 - 1)))].x;
            if (b > 0 && b < P2 - b) acc += ACC[padded(j * P2 + P2 - b)].x;
        }
        hblk[jb.hoff + k] = acc * inv;
    }
}

// The forward half of the apply's fft_1d_x2 alone: the same passes, the span-1 pass without the
// spectrum product and the inverse. The result is in bit-reversed order (element e
// holds frequency brev(e) of both of its complex values).
template <int RL>
__device__ __forceinline__ void bottom_fwd_1d_x2(ulonglong2 *Z, int NP, int nplane, int ln) {
    constexpr int R = 1 << RL;
    const int glog = ln - RL;
    const int total = nplane << glog;
    const int gmask = (1 << glog) - 1;
    for (int w = threadIdx.x; w < total; w += blockDim.x) {
        const int g = w & gmask, p = w >> glog;
        const int e0 = g << RL;
        ulonglong2 *Zp = Z + p * NP;
        int adr[R];
        dev::slots_1d<RL, 0>(e0, adr);
        dev::Cx2 v[R];
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const ulonglong2 q = Zp[adr[t]];
            v[t] = dev::Cx2{q.x, q.y};
        }
        dev::dft_dif_x2<RL>(v);
#pragma unroll
        for (int t = 0; t < R; ++t) Zp[adr[t]] = make_ulonglong2(v[t].re, v[t].im);
    }
    __syncthreads();
}

__device__ __forceinline__ void fwd_1d_x2(ulonglong2 *Z, int NP, int nplane, int ln, const float2 *__restrict__ tw,
                                          const ulonglong2 *__restrict__ twb) {
    const int full = ln / 3, rem = ln - 3 * full;
    if (full > 0) {
        if (rem == 2) dev::pass_1d_dispatch<false, 2>(Z, NP, nplane, ln, ln - 2, tw, twb);
        else if (rem == 1) dev::pass_1d_dispatch<false, 1>(Z, NP, nplane, ln, ln - 1, tw, twb);
        for (int k = 0; k < full - 1; ++k) dev::pass_1d_dispatch<false, 3>(Z, NP, nplane, ln, ln - rem - 3 * (k + 1), tw, twb);
        bottom_fwd_1d_x2<3>(Z, NP, nplane, ln);
    } else if (rem == 2) {
        bottom_fwd_1d_x2<2>(Z, NP, nplane, ln);
    } else {
        bottom_fwd_1d_x2<1>(Z, NP, nplane, ln);
    }
}

// One-dimensional FFT jobs (lp2 = 0) on the paired-FP32 transforms of the apply: one CTA per
// job and block of kGradCB channels, as grad_fft_kernel, but two channels per transform: the
// element of depth r holds z_c = gsum_c + i fsum_c for channels c and c + 1 (lane pairs), and the
// forward transform of fwd_1d_x2 gives both spectra at once. Per channel the correlation spectrum
// is A^ B^ = (z(f)^2 - conj z(-f)^2) / 4i, summed over the block's channels (in channel order)
// into ACC; then, as in grad_fft_kernel, the inverse transform and the binning along depth.
// Shared memory: NP 16-byte elements and padded_size(NP) complex accumulators.
__global__ void __launch_bounds__(256) grad_fft1d_x2_kernel(const GradJob *__restrict__ jobs,
                                                            const int32_t *__restrict__ ids,
                                                            const int32_t *__restrict__ key_r, int d,
                                                            const float *__restrict__ gsum,
                                                            const float *__restrict__ fsum,
                                                            const float2 *__restrict__ tw,
                                                            const ulonglong2 *__restrict__ twb,
                                                            float *__restrict__ hist) {
    extern __shared__ ulonglong2 gzx[];
    const GradJob jb = jobs[ids[blockIdx.x]];
    const int ln = jb.lp1, NP = 1 << ln;
    const int padnp = padded_size(NP);
    ulonglong2 *Zx = gzx;
    float2 *ACC = reinterpret_cast<float2 *>(gzx + NP);
    for (int i = threadIdx.x; i < padnp; i += blockDim.x) ACC[i] = make_float2(0.f, 0.f);
    const int nk = jb.ke - jb.kb;
    const int cb0 = blockIdx.y * kGradCB, cb1 = min(d, cb0 + kGradCB);
    for (int c = cb0; c < cb1; c += 2) {
        const bool two = c + 1 < cb1;
        for (int i = threadIdx.x; i < NP; i += blockDim.x) Zx[i] = make_ulonglong2(0ull, 0ull);
        __syncthreads();
        for (int t = threadIdx.x; t < nk; t += blockDim.x) {
            const int64_t k = jb.kb + t;
            const float g0 = gsum[k * d + c], f0 = fsum[k * d + c];
            const float g1 = two ? gsum[k * d + c + 1] : 0.f, f1 = two ? fsum[k * d + c + 1] : 0.f;
            Zx[dev::swz(key_r[k])] = make_ulonglong2(dev::vpack(g0, g1), dev::vpack(f0, f1));
        }
        __syncthreads();
        fwd_1d_x2(Zx, NP, 1, ln, tw, twb);
        for (int e = threadIdx.x; e < NP; e += blockDim.x) {
            const int f = brev_bits(e, ln), q = brev_bits((NP - f) & (NP - 1), ln);
            const ulonglong2 a = Zx[dev::swz(e)], b = Zx[dev::swz(q)];
            float zr0, zr1, zi0, zi1, wr0, wr1, wi0, wi1;
            dev::vunpack(a.x, zr0, zr1);
            dev::vunpack(a.y, zi0, zi1);
            dev::vunpack(b.x, wr0, wr1);
            dev::vunpack(b.y, wi0, wi1);
            // z^2 - conj(w)^2 per channel: real (zr^2 - zi^2) - (wr^2 - wi^2), imaginary 2 zr zi + 2 wr wi
            const float re0 = (zr0 * zr0 - zi0 * zi0) - (wr0 * wr0 - wi0 * wi0);
            const float im0 = 2.f * (zr0 * zi0 + wr0 * wi0);
            const float re1 = (zr1 * zr1 - zi1 * zi1) - (wr1 * wr1 - wi1 * wi1);
            const float im1 = 2.f * (zr1 * zi1 + wr1 * wi1);
            // / (4 i): (im, -re) / 4; channel c first, then c + 1
            float2 acc = ACC[padded(e)];
            acc.x += 0.25f * im0;
            acc.y += -0.25f * re0;
            if (two) {
                acc.x += 0.25f * im1;
                acc.y += -0.25f * re1;
            }
            ACC[padded(e)] = acc;
        }
        __syncthreads();
    }
    dev::fft_axis<true>(ACC, padnp, 1, ln, 1, 0, 1, true, tw, false);
    __syncthreads();
    const float inv = 1.f / float(NP);
    const int K = 2 * jb.maxr + 1;
    float *hblk = hist + int64_t(blockIdx.y) * K;
    for (int k = threadIdx.x; k < K; k += blockDim.x) hblk[jb.hoff + k] = ACC[padded(k)].x * inv;
}

// The job's histogram (block 0's slot) = its first nblk channel blocks' histograms added in block order.
__global__ void grad_block_reduce(const GradJob *__restrict__ jobs, int n_jobs, int nblk, float *__restrict__ hist) {
    const GradJob jb = jobs[blockIdx.x];
    if (jb.mode != 0) return;
    const int K = 2 * jb.maxr + jb.maxx + 1;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        float acc = hist[jb.hoff + k];
        for (int b = 1; b < nblk; ++b) acc += hist[jb.hoff + int64_t(b) * K + k];
        hist[jb.hoff + k] = acc;
    }
}

// Direct jobs, pass 1: M[i][l] = <gsum_i, fsum_l> over the d channels for all
// pairs of the job's bins, a small nk x nk x d product: one CTA per (job, 32 x 32
// tile, block of kGradDotCB channels; blockIdx.y), channels streamed through
// shared memory in chunks of 32 (fixed order). Each channel block writes its own
// partial product, at moff + blockIdx.y * nk * nk.
constexpr int kGradDotCB = 512;

__global__ void __launch_bounds__(256) grad_pair_dots(const GradJob *__restrict__ jobs,
                                                      const int64_t *__restrict__ items, int d,
                                                      const float *__restrict__ gsum, const float *__restrict__ fsum,
                                                      float *__restrict__ M) {
    __shared__ float As[32][33], Bs[32][33];
    const int64_t it = items[blockIdx.x];  // job index << 16 | tile index (ti << 8 | tl)
    const GradJob jb = jobs[it >> 16];
    const int nk = jb.ke - jb.kb;
    const int i0 = int((it >> 8) & 255) * 32, l0 = int(it & 255) * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // ty: 0..7, four rows each
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    const int cb0 = blockIdx.y * kGradDotCB, cb1 = min(d, cb0 + kGradDotCB);
    for (int c0 = cb0; c0 < cb1; c0 += 32) {
        for (int q = threadIdx.x; q < 32 * 32; q += 256) {
            const int r = q >> 5, c = q & 31;
            const bool cok = c0 + c < cb1;
            As[r][c] = (i0 + r < nk && cok) ? gsum[int64_t(jb.kb + i0 + r) * d + c0 + c] : 0.f;
            Bs[r][c] = (l0 + r < nk && cok) ? fsum[int64_t(jb.kb + l0 + r) * d + c0 + c] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int c = 0; c < 32; ++c) {
            const float b = Bs[tx][c];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = fmaf(As[ty * 4 + u][c], b, acc[u]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int i = i0 + ty * 4 + u, l = l0 + tx;
        if (i < nk && l < nk) M[jb.moff + int64_t(blockIdx.y) * nk * nk + int64_t(i) * nk + l] = acc[u];
    }
}

// Direct jobs, pass 2: M[i][l] = sum of the ncb channel blocks' partials (in
// block order), then H[k] = sum over pairs (i, l) in order with
// r_i + r_l + |x_i - x_l| = k of M[i][l]; one CTA per job, one thread per k.
__global__ void grad_direct_bin(const GradJob *__restrict__ jobs, const int32_t *__restrict__ djobs, int ncb,
                                const int32_t *__restrict__ key_r, const int32_t *__restrict__ key_x,
                                float *__restrict__ M, float *__restrict__ hist) {
    const GradJob jb = jobs[djobs[blockIdx.x]];
    const int nk = jb.ke - jb.kb;
    const int K = 2 * jb.maxr + jb.maxx + 1;
    const int64_t nn = int64_t(nk) * nk;
    for (int64_t q = threadIdx.x; q < nn; q += blockDim.x) {
        float acc = M[jb.moff + q];
        for (int b = 1; b < ncb; ++b) acc += M[jb.moff + b * nn + q];
        M[jb.moff + q] = acc;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        float acc = 0.f;
        for (int i = 0; i < nk; ++i) {
            const int ri = __ldg(key_r + jb.kb + i), xi = __ldg(key_x + jb.kb + i);
            if (ri > k) continue;
            for (int l = 0; l < nk; ++l) {
                const int dd = ri + __ldg(key_r + jb.kb + l) + abs(xi - __ldg(key_x + jb.kb + l));
                if (dd == k) acc += M[jb.moff + int64_t(i) * nk + l];
            }
        }
        hist[jb.hoff + k] = acc;
    }
}

// Direct jobs, pass 2 in one sweep over the pairs: M[i][l] = sum of the ncb channel blocks'
// partials (in block order), then every pair adds M[i][l] into a shared-memory histogram of
// 64-bit fixed-point integers at r_i + r_l + |x_i - x_l| (exact, so the order of the atomic adds
// does not matter), with the scale 2^S, S = 61 - ceil(log2 nk^2) - ceil(log2 max |M|), that no sum
// can overflow. The job's keys are staged in shared memory. One CTA per job; the plan uses it when
// its histograms and keys fit (8 K + 8 nk bytes).
__host__ __device__ inline size_t grad_direct_bin_smem(int max_k, int max_nk) {
    return size_t((max_k + 1) & ~1) * 8 + size_t(max_nk) * 8 + 64;
}

__global__ void __launch_bounds__(256) grad_direct_bin_fx(const GradJob *__restrict__ jobs,
                                                          const int32_t *__restrict__ djobs, int ncb,
                                                          const int32_t *__restrict__ key_r,
                                                          const int32_t *__restrict__ key_x, int max_k,
                                                          float *__restrict__ M, float *__restrict__ hist) {
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned long long shd[];
    __shared__ float s_max[8];
    const GradJob jb = jobs[djobs[blockIdx.x]];
    const int nk = jb.ke - jb.kb;
    const int K = 2 * jb.maxr + jb.maxx + 1;
    const int64_t nn = int64_t(nk) * nk;
    unsigned long long *h64 = shd;
    int *sr = reinterpret_cast<int *>(shd + ((max_k + 1) & ~1)), *sx = sr + nk;
    for (int k = threadIdx.x; k < K; k += blockDim.x) h64[k] = 0ull;
    for (int i = threadIdx.x; i < nk; i += blockDim.x) {
        sr[i] = key_r[jb.kb + i];
        sx[i] = key_x[jb.kb + i];
    }
    float mx = 0.f;
    for (int64_t q = threadIdx.x; q < nn; q += blockDim.x) {
        float acc = M[jb.moff + q];
        for (int b = 1; b < ncb; ++b) acc += M[jb.moff + b * nn + q];
        M[jb.moff + q] = acc;
        mx = fmaxf(mx, fabsf(acc));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, o));
    if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = 0.f;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) mx = fmaxf(mx, s_max[w]);
    int S = 0;
    if (mx > 0.f) {
        int e;
        frexpf(mx, &e);                                              // mx < 2^e
        const int ln2 = 64 - __clzll(static_cast<unsigned long long>(nn));   // nn < 2^ln2
        S = 61 - ln2 - e;
    }
    const float sc1 = ldexpf(1.f, S / 2), sc2 = ldexpf(1.f, S - S / 2);
    for (int64_t q = threadIdx.x; q < nn; q += blockDim.x) {
        const int i = int(q / nk), l = int(q - int64_t(i) * nk);
        const int D = sr[i] + sr[l] + abs(sx[i] - sx[l]);
        const float v = M[jb.moff + q];
        if (D < K && v != 0.f) atomicAdd(&h64[D], static_cast<unsigned long long>(__float2ll_rn(v * sc1 * sc2)));
    }
    __syncthreads();
    const float inv1 = ldexpf(1.f, -(S / 2)), inv2 = ldexpf(1.f, -(S - S / 2));
    for (int k = threadIdx.x; k < K; k += blockDim.x)
        hist[jb.hoff + k] = float(static_cast<long long>(h64[k])) * inv1 * inv2;
}

template <typename T>
__device__ __forceinline__ float ldf(const T *p);
template <>
__device__ __forceinline__ float ldf<float>(const float *p) { return *p; }
template <>
__device__ __forceinline__ float ldf<__nv_bfloat16>(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

// Leaves, pass 1: for every ordered pair (i, j) of a leaf, its distance and
// <g_i, F_j>, at pair_off[leaf] + (i - lo) * s + (j - lo). One warp per pair at a
// time: lanes take channels 32 apart, then a butterfly of shuffles (fixed order)
// adds the lanes' partial sums.
template <typename T>
__global__ void grad_leaf_pairs(const int32_t *__restrict__ leaf_ptr, const int64_t *__restrict__ pair_off,
                                const int32_t *__restrict__ leaf_vtx, const int32_t *__restrict__ leaf_dist,
                                const int32_t *__restrict__ leaf_pdist, const T *__restrict__ G,
                                const T *__restrict__ F, int d, float *__restrict__ pval, int32_t *__restrict__ pdst) {
    const int lf = blockIdx.x;
    const int lo = leaf_ptr[lf], hi = leaf_ptr[lf + 1], s = hi - lo;
    const int64_t base = pair_off[lf];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t q = warp; q < int64_t(s) * s; q += nw) {
        const int ii = int(q / s), jj = int(q - int64_t(ii) * s);
        const int i = lo + ii, j = lo + jj;
        // dhat(i, j) = D(i) + D(j) - 2 min over (min(i, j), max(i, j)] of the parent distances
        int dist = 0;
        if (i != j) {
            int m = 0x7fffffff;
            for (int w = min(i, j) + 1 + lane; w <= max(i, j); w += 32) m = min(m, leaf_pdist[w]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
            dist = leaf_dist[i] + leaf_dist[j] - 2 * m;
        }
        const int64_t vi = leaf_vtx[i], vj = leaf_vtx[j];
        float acc = 0.f;
        for (int c = lane; c < d; c += 32) acc = fmaf(ldf<T>(G + vi * d + c), ldf<T>(F + vj * d + c), acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            pval[base + q] = acc;
            pdst[base + q] = dist;
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

// Leaves in one pass: one CTA per leaf (and group of channel blocks), eight warps, each warp a block of 32
// targets (one per lane) against every source of the leaf, the channels in blocks
// of 16 (the histogram is linear in the channels, so the blocks add up). The
// pair distances follow the leaf walk of the apply: dhat(i, j) = D(i) + D(j) -
// 2 m(i, j) with running minima m over the parent distances, the sources inside
// the block in an ascending and a descending sweep, the sources after it
// ascending from the block's suffix minima, those before it descending from its
// prefix minima. The pair values <g_i, F_j> are added into one histogram of
// 64-bit fixed-point integers in shared memory: integer addition is exact and
// associative, so the result does not depend on the order of the atomic adds
// (deterministic), and the scale 2^S is chosen per leaf so that no sum can
// overflow: |<g_i, F_j>| <= max ||g|| max ||F|| = B, at most n^2 pairs, so
// S = 61 - ceil(log2 n^2) - ceil(log2 B) keeps every partial sum below 2^61;
// each value is rounded once to a multiple of 2^-S (<= 2^-S / 2 from exact).
constexpr int kGradLeafWarps = 8;

// The scale exponent S of each leaf (above), from the largest squared row norms of g and F over
// the leaf's vertices (all channels): one CTA per leaf.
template <typename T>
__global__ void grad_leaf_scale(const int32_t *__restrict__ leaf_ptr, const int32_t *__restrict__ leaf_vtx,
                                const T *__restrict__ G, const T *__restrict__ F, int d, int32_t *__restrict__ S_out) {
    constexpr unsigned FULL = 0xffffffffu;
    __shared__ float s_max[2][32];
    const int lf = blockIdx.x;
    const int lo = leaf_ptr[lf], n = leaf_ptr[lf + 1] - lo;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float mg = 0.f, mf = 0.f;
    for (int i = warp; i < n; i += nw) {   // one warp per vertex, lanes over the channels
        const int64_t v = leaf_vtx[lo + i];
        float sg = 0.f, sf = 0.f;
        for (int c = lane; c < d; c += 32) {
            const float a = ldf<T>(G + v * d + c), b = ldf<T>(F + v * d + c);
            sg = fmaf(a, a, sg);
            sf = fmaf(b, b, sf);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sg += __shfl_xor_sync(FULL, sg, o);
            sf += __shfl_xor_sync(FULL, sf, o);
        }
        mg = fmaxf(mg, sg);
        mf = fmaxf(mf, sf);
    }
    if (lane == 0) {
        s_max[0][warp] = mg;
        s_max[1][warp] = mf;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; ++w) {
            mg = fmaxf(mg, s_max[0][w]);
            mf = fmaxf(mf, s_max[1][w]);
        }
        // B^2 = mg mf (the squared sums round up by at most a few ulps, covered by the margin)
        int S = 0;
        if (mg > 0.f && mf > 0.f) {
            int eg, ef;
            frexpf(mg, &eg);   // mg < 2^eg
            frexpf(mf, &ef);
            const int lb = (eg + ef + 1) / 2 + 1;          // B < 2^lb
            const int ln2 = 2 * (32 - __clz(max(n, 1)));   // n^2 <= 2^ln2
            S = 61 - ln2 - lb;
        }
        S_out[lf] = S;
    }
}

// Leaves whose channel blocks were split over several CTAs: their exact integer sums, scaled
// back by 2^-S, one CTA per leaf.
// h64 holds the leaves' histograms from offset h64_base of hist (the leaves follow the jobs).
__global__ void grad_leaf_h64_to_float(const int32_t *__restrict__ S_in, const int64_t *__restrict__ hist_off,
                                       const int32_t *__restrict__ hist_len,
                                       const unsigned long long *__restrict__ h64, int64_t h64_base,
                                       float *__restrict__ hist) {
    const int lf = blockIdx.x, S = S_in[lf];
    const float inv1 = ldexpf(1.f, -(S / 2)), inv2 = ldexpf(1.f, -(S - S / 2));
    const int64_t off = hist_off[lf];
    for (int k = threadIdx.x; k < hist_len[lf]; k += blockDim.x)
        hist[off + k] = float(static_cast<long long>(h64[off - h64_base + k])) * inv1 * inv2;
}

// the fixed-point histogram rounded up to an even count of 8-byte entries, so that the source
// rows after it start on a 16-byte boundary (they are read as float4)
__host__ __device__ inline int grad_leaf_hist_slots(int max_hl) { return (max_hl + 1) & ~1; }

__host__ __device__ inline size_t grad_leaf_warp_smem(int max_n, int max_hl) {
    return size_t(grad_leaf_hist_slots(max_hl)) * 8 + size_t(max_n) * 16 * 4 + size_t(2 * max_n + 2) * 4 + 64;
}

template <typename T>
__global__ void __launch_bounds__(32 * kGradLeafWarps) grad_leaf_warp_hist(
    const int32_t *__restrict__ leaf_ptr, const int64_t *__restrict__ hist_off, const int32_t *__restrict__ hist_len,
    const int32_t *__restrict__ leaf_vtx, const int32_t *__restrict__ leaf_dist, const int32_t *__restrict__ leaf_pdist,
    const T *__restrict__ G, const T *__restrict__ F, int d, int max_n, int max_hl,
    const int32_t *__restrict__ S_in, unsigned long long *__restrict__ h64_out, int64_t h64_base,
    float *__restrict__ hist) {
    constexpr int INF = 0x7fffffff;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned long long smh[];
    const int lf = blockIdx.x;
    const int lo = leaf_ptr[lf], n = leaf_ptr[lf + 1] - lo, hl = hist_len[lf];
    unsigned long long *h64 = smh;                                       // max_hl fixed-point sums
    float *sx = reinterpret_cast<float *>(smh + grad_leaf_hist_slots(max_hl));   // the block's source rows
    int *sdist = reinterpret_cast<int *>(sx + max_n * 16), *spd = sdist + max_n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        sdist[i] = leaf_dist[lo + i];
        spd[i] = leaf_pdist[lo + i];
    }
    if (threadIdx.x == 0) spd[n] = INF;
    for (int k = threadIdx.x; k < hl; k += blockDim.x) h64[k] = 0ull;
    const int S = S_in[lf];
    const float sc1 = ldexpf(1.f, S / 2), sc2 = ldexpf(1.f, S - S / 2);  // 2^S in two representable factors
    auto add = [&](int D, float v) {
        if (D >= 0 && D < hl) atomicAdd(&h64[D], static_cast<unsigned long long>(__float2ll_rn(v * sc1 * sc2)));
    };
    // this CTA's channel blocks: blockIdx.y, + gridDim.y, ...
    for (int c0 = 16 * blockIdx.y; c0 < d; c0 += 16 * gridDim.y) {
        __syncthreads();
        for (int q = threadIdx.x; q < n * 16; q += blockDim.x) {
            const int j = q >> 4, c = q & 15;
            sx[q] = c0 + c < d ? ldf<T>(F + int64_t(leaf_vtx[lo + j]) * d + c0 + c) : 0.f;
        }
        __syncthreads();
        // work units: (target block, part), part 0 the sources inside the block and after it, part 1
        // those before it, so that a leaf of few blocks still keeps the eight warps busy
        const int nblk = (n + 31) / 32;
        for (int u = warp; u < 2 * nblk; u += kGradLeafWarps) {
            const int a = (u >> 1) * 32, part = u & 1;
            if (part == 1 && a == 0) continue;   // nothing before the first block (warp-uniform)
            const int bend = min(a + 32, n);
            const int ti = a + lane;
            const bool act = ti < n;
            const int Di = act ? sdist[ti] : 0;
            float g[16];
            {
                const int64_t vi = act ? leaf_vtx[lo + ti] : 0;
#pragma unroll
                for (int c = 0; c < 16; ++c) g[c] = (act && c0 + c < d) ? ldf<T>(G + vi * d + c0 + c) : 0.f;
            }
            // <g_i, x_j> as paired FP32 FMAs: lanes (even, odd channels), added at the end
            dev::f32x2 gp[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) gp[c] = dev::vpack(g[2 * c], g[2 * c + 1]);
            auto dot = [&](int j) {
                const float4 *x = reinterpret_cast<const float4 *>(sx + j * 16);
                dev::f32x2 s = 0ull;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 r = x[q];
                    s = dev::vfma(gp[2 * q], dev::vpack(r.x, r.y), s);
                    s = dev::vfma(gp[2 * q + 1], dev::vpack(r.z, r.w), s);
                }
                float s0, s1;
                dev::vunpack(s, s0, s1);
                return s0 + s1;
            };
            // carries: suffix min over (i, bend - 1], prefix min over (a, i]
            int suf = (a + lane + 1 < bend) ? spd[a + lane + 1] : INF;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_down_sync(FULL, suf, o);
                if (lane + o < 32) suf = min(suf, u);
            }
            int pre = (lane > 0 && a + lane < bend) ? spd[a + lane] : INF;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(FULL, pre, o);
                if (lane >= o) pre = min(pre, u);
            }
            int m = INF;
            if (part == 0) {
            // sources inside the block: ascending for j >= i (j = i at distance 0), descending for j < i
            for (int j = a; j < bend; ++j) {
                if (j > ti) m = min(m, spd[j]);
                add(!act || j < ti ? -1 : j == ti ? 0 : Di + sdist[j] - 2 * m, dot(j));
            }
            m = INF;
            for (int j = bend - 1; j >= a; --j) {
                if (j < ti) m = min(m, spd[j + 1]);
                add(act && j < ti ? Di + sdist[j] - 2 * m : -1, dot(j));
            }
            // sources after the block, ascending
            m = suf;
            for (int j = bend; j < n; ++j) {
                m = min(m, spd[j]);
                add(act ? Di + sdist[j] - 2 * m : -1, dot(j));
            }
            } else {
            // sources before the block, descending
            m = pre;
            for (int j = a - 1; j >= 0; --j) {
                m = min(m, spd[j + 1]);
                add(act ? Di + sdist[j] - 2 * m : -1, dot(j));
            }
            }
        }
    }
    __syncthreads();
    if (gridDim.y == 1) {
        float *out = hist + hist_off[lf];
        const float inv1 = ldexpf(1.f, -(S / 2)), inv2 = ldexpf(1.f, -(S - S / 2));
        for (int k = threadIdx.x; k < hl; k += blockDim.x)
            out[k] = float(static_cast<long long>(h64[k])) * inv1 * inv2;
    } else {
        // exact integer sums of the channel-block CTAs (zeroed beforehand), converted afterwards
        unsigned long long *out = h64_out + (hist_off[lf] - h64_base);
        for (int k = threadIdx.x; k < hl; k += blockDim.x)
            if (h64[k]) atomicAdd(out + k, h64[k]);
    }
}

// C[k] = sum over segments (fixed order) of sign * hist_segment[k], in FP64. One
// warp per k: lanes take segments 32 apart, then a butterfly of shuffles (fixed
// order) adds the lanes' partial sums. The segments come sorted by length, longest
// first, so those with an entry k are a prefix, found by bisection: the work is the
// total histogram length, not segments x lengths.
__global__ void grad_reduce(int n_seg, const int64_t *__restrict__ seg_off, const int32_t *__restrict__ seg_len,
                            const float *__restrict__ seg_sign, const float *__restrict__ hist, int64_t len,
                            double *__restrict__ C) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t k = blockIdx.x * int64_t(blockDim.x >> 5) + (threadIdx.x >> 5); k < len; k += warps) {
        int lo = 0, hi = n_seg;   // the segments with seg_len > k: [0, lo)
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (seg_len[mid] > k) lo = mid + 1;
            else hi = mid;
        }
        double acc = 0.0;
        for (int sgm = lane; sgm < lo; sgm += 32) acc += double(seg_sign[sgm]) * double(hist[seg_off[sgm] + k]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) C[k] = acc;
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
