// Device kernels of the StAd-TFI apply (sm_103a).
//
// One apply evaluates every recursive call of the plan at once: the cross
// terms of different calls depend only on the input field (Eq. "stad-split",
// Algorithm 5), so there is no level-by-level dependency on the device.
//
//   leaf_kernel    dense leaf calls: w^(S) = f(D_S) x_S (base case of Algorithm 5
//                  generalised to |V(S)| <= s0), distances from a sparse-table
//                  range minimum over the leaf's preorder
//   bucket_kernel  segmented sums of field rows into the occupied bins: the
//                  aggregates A_r[t] (Section 2.2) and the profiles b_alpha[r]
//                  (Eq. "stad-E"), in plan order (deterministic, no atomics)
//   fft_kernel     per job, the table G = K * A (Eq. "stad-2d-convolution") or a
//                  correction E_alpha (Eq. "stad-E") as a circular FFT
//                  correlation in shared memory: in-place radix-2 DIF forward
//                  (natural -> bit-reversed), product with the cached kernel
//                  spectrum (stored bit-reversed), DIT inverse (bit-reversed ->
//                  natural); two channels ride in one complex transform
//   direct_kernel  the same jobs by direct summation over occupied bins
//   gather_kernel  out[u] = leaf term + sum over u's calls of
//                  G_{d(u)}[X(pi u)] - E_alpha[d(u)] (Lemma "Cross-component
//                  correction"), one write per output row
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace tfi {
namespace dev {

constexpr int kTwLogDev = 14;

struct FftItem {
    int32_t job;
    int32_t pair0;
    int32_t npair;
};

struct DirItem {
    int32_t job;
    int32_t q0;
};

struct JobDev {
    int32_t kb, ke;
    int32_t lp1, lp2;
    int32_t spec_off;  // in complex elements
    int32_t pad;
};

template <typename T>
__device__ __forceinline__ float to_f(T v);
template <>
__device__ __forceinline__ float to_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T>
__device__ __forceinline__ T from_f(float v);
template <>
__device__ __forceinline__ float from_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// ---------------------------------------------------------------------------
// bucket: kbuf[k, c] = sum_{v in bin k} F[v, c]
// ---------------------------------------------------------------------------
template <typename T, int V>
__global__ void bucket_kernel(int64_t n_keys, const int32_t *__restrict__ key_ptr, const int32_t *__restrict__ key_vtx,
                              const T *__restrict__ F, int d, float *__restrict__ kbuf) {
    const int chunks = d / V;
    const int64_t total = n_keys * chunks;
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
        const int64_t k = t / chunks;
        const int c = int(t - k * chunks) * V;
        float acc[V];
#pragma unroll
        for (int i = 0; i < V; ++i) acc[i] = 0.f;
        const int e1 = key_ptr[k + 1];
        for (int e = key_ptr[k]; e < e1; ++e) {
            const T *row = F + int64_t(key_vtx[e]) * d + c;
#pragma unroll
            for (int i = 0; i < V; ++i) acc[i] += to_f<T>(row[i]);
        }
        float *dst = kbuf + k * d + c;
#pragma unroll
        for (int i = 0; i < V; ++i) dst[i] = acc[i];
    }
}

// ---------------------------------------------------------------------------
// FFT job kernel
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// Radix-2 passes along one axis of npair arrays of NP points each.
// Axis of length n = 2^ln with element stride `stride`; the other axis has
// `lines` lines with stride `lstride`. rows: stride 1, lstride n. cols: stride
// lines, lstride 1 (consecutive threads take consecutive columns).
template <bool INVERSE>
__device__ __forceinline__ void fft_axis(float2 *Z, int npair, int lnp, int ln, int stride, int lines, int lstride,
                                         bool cols, const float2 *__restrict__ tw) {
    if (ln == 0) return;
    const int NP = 1 << lnp;
    const int half_np = NP >> 1;
    const int nb = npair * half_np;
    const int hn = 1 << (ln - 1);  // butterflies per line
    for (int s = 0; s < ln; ++s) {
        const int lh = INVERSE ? s : (ln - 1 - s);  // log2(half)
        const int half = 1 << lh;
        const int twshift = kTwLogDev - 1 - lh;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            const int p = b >> (lnp - 1);
            const int bb = b & (half_np - 1);
            int line, k;
            if (cols) {
                line = bb & (lines - 1);
                k = bb / lines;
            } else {
                line = bb >> (ln - 1);
                k = bb & (hn - 1);
            }
            const int j = k & (half - 1);
            const int i0 = ((k >> lh) << (lh + 1)) + j;
            float2 *base = Z + p * NP + line * lstride;
            float2 *a0 = base + i0 * stride;
            float2 *a1 = a0 + half * stride;
            const float2 w = __ldg(tw + (j << twshift));
            const float2 u = *a0, v = *a1;
            if (!INVERSE) {
                *a0 = make_float2(u.x + v.x, u.y + v.y);
                *a1 = cmul(make_float2(u.x - v.x, u.y - v.y), w);
            } else {
                const float2 t = cmulc(v, w);
                *a0 = make_float2(u.x + t.x, u.y + t.y);
                *a1 = make_float2(u.x - t.x, u.y - t.y);
            }
        }
        __syncthreads();
    }
}

__global__ void fft_kernel(const FftItem *__restrict__ items, const JobDev *__restrict__ jobs,
                           const int32_t *__restrict__ key_r, const int32_t *__restrict__ key_x, int d,
                           const float *__restrict__ kbuf, float *__restrict__ vbuf,
                           const float2 *__restrict__ spectra, const float2 *__restrict__ tw) {
    extern __shared__ float2 Z[];
    const FftItem it = items[blockIdx.x];
    const JobDev jb = jobs[it.job];
    const int lp1 = jb.lp1, lp2 = jb.lp2, lnp = lp1 + lp2;
    const int NP = 1 << lnp, P1 = 1 << lp1, P2 = 1 << lp2;
    const int npair = it.npair;
    for (int i = threadIdx.x; i < npair * NP; i += blockDim.x) Z[i] = make_float2(0.f, 0.f);
    __syncthreads();
    const int nk = jb.ke - jb.kb;
    // scatter bin sums; depth reversed so the depth correlation becomes a convolution
    for (int t = threadIdx.x; t < nk * npair; t += blockDim.x) {
        const int kk = t / npair, p = t - kk * npair;
        const int k = jb.kb + kk;
        const int ch = 2 * (it.pair0 + p);
        const float re = kbuf[int64_t(k) * d + ch];
        const float im = (ch + 1 < d) ? kbuf[int64_t(k) * d + ch + 1] : 0.f;
        const int pos = ((P1 - key_r[k]) & (P1 - 1)) * P2 + key_x[k];
        Z[p * NP + pos] = make_float2(re, im);
    }
    __syncthreads();
    fft_axis<false>(Z, npair, lnp, lp2, 1, P1, P2, false, tw);   // rows: backbone axis
    fft_axis<false>(Z, npair, lnp, lp1, P2, P2, 1, true, tw);    // columns: depth axis
    const float2 *S = spectra + jb.spec_off;
    for (int i = threadIdx.x; i < npair * NP; i += blockDim.x) Z[i] = cmul(Z[i], __ldg(S + (i & (NP - 1))));
    __syncthreads();
    fft_axis<true>(Z, npair, lnp, lp1, P2, P2, 1, true, tw);
    fft_axis<true>(Z, npair, lnp, lp2, 1, P1, P2, false, tw);
    for (int t = threadIdx.x; t < nk * npair; t += blockDim.x) {
        const int kk = t / npair, p = t - kk * npair;
        const int k = jb.kb + kk;
        const int ch = 2 * (it.pair0 + p);
        const float2 v = Z[p * NP + key_r[k] * P2 + key_x[k]];
        vbuf[int64_t(k) * d + ch] = v.x;
        if (ch + 1 < d) vbuf[int64_t(k) * d + ch + 1] = v.y;
    }
}

// ---------------------------------------------------------------------------
// direct job kernel: one warp per (job, 32 query bins), CH channels per pass
// ---------------------------------------------------------------------------
template <int CH, int WARPS>
__global__ void direct_kernel(const DirItem *__restrict__ items, int n_items, const JobDev *__restrict__ jobs,
                              const int32_t *__restrict__ key_r, const int32_t *__restrict__ key_x, int d,
                              const float *__restrict__ kbuf, float *__restrict__ vbuf, const float *__restrict__ ftab) {
    __shared__ int sr[WARPS][32];
    __shared__ int sx[WARPS][32];
    __shared__ float sv[WARPS][32][CH];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int w = blockIdx.x * WARPS + warp;
    if (w >= n_items) return;
    const int c0 = blockIdx.y * CH;
    const DirItem it = items[w];
    const JobDev jb = jobs[it.job];
    const int i = it.q0 + lane;
    const bool valid = i < jb.ke;
    const int ri = valid ? key_r[i] : 0;
    const int xi = valid ? key_x[i] : 0;
    float acc[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) acc[c] = 0.f;
    for (int s0 = jb.kb; s0 < jb.ke; s0 += 32) {
        const int j = s0 + lane;
        if (j < jb.ke) {
            sr[warp][lane] = key_r[j];
            sx[warp][lane] = key_x[j];
#pragma unroll
            for (int c = 0; c < CH; ++c) sv[warp][lane][c] = (c0 + c < d) ? kbuf[int64_t(j) * d + c0 + c] : 0.f;
        }
        __syncwarp();
        const int cnt = min(32, jb.ke - s0);
        for (int t = 0; t < cnt; ++t) {
            const float f = __ldg(ftab + ri + sr[warp][t] + abs(xi - sx[warp][t]));
#pragma unroll
            for (int c = 0; c < CH; ++c) acc[c] = fmaf(f, sv[warp][t][c], acc[c]);
        }
        __syncwarp();
    }
    if (valid) {
#pragma unroll
        for (int c = 0; c < CH; ++c)
            if (c0 + c < d) vbuf[int64_t(i) * d + c0 + c] = acc[c];
    }
}

// ---------------------------------------------------------------------------
// gather: out[u] = leaf[u] + sum_calls (val[A-bin] - val[b-bin])
// ---------------------------------------------------------------------------
template <typename T, int V>
__global__ void gather_kernel(int n, const int32_t *__restrict__ vrec_ptr, const int32_t *__restrict__ akey,
                              const int32_t *__restrict__ bkey, const float *__restrict__ vbuf,
                              const float *__restrict__ leaf, const uint8_t *__restrict__ in_leaf, int d,
                              T *__restrict__ out) {
    const int chunks = d / V;
    const int64_t total = int64_t(n) * chunks;
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
        const int64_t u = t / chunks;
        const int c = int(t - u * chunks) * V;
        float acc[V];
        const bool has_leaf = in_leaf[u] != 0;
#pragma unroll
        for (int i = 0; i < V; ++i) acc[i] = has_leaf ? leaf[u * d + c + i] : 0.f;
        const int e1 = vrec_ptr[u + 1];
        for (int e = vrec_ptr[u]; e < e1; ++e) {
            const float *g = vbuf + int64_t(akey[e]) * d + c;
#pragma unroll
            for (int i = 0; i < V; ++i) acc[i] += g[i];
            const int b = bkey[e];
            if (b >= 0) {
                const float *h = vbuf + int64_t(b) * d + c;
#pragma unroll
                for (int i = 0; i < V; ++i) acc[i] -= h[i];
            }
        }
#pragma unroll
        for (int i = 0; i < V; ++i) out[u * d + c + i] = from_f<T>(acc[i]);
    }
}

// ---------------------------------------------------------------------------
// dense leaves: one CTA per leaf group, CH channels per pass
// dhat(i, j) = D(i) + D(j) - 2 min_{w in (i, j]} D(parent(w)) in preorder
// ---------------------------------------------------------------------------
template <typename T, int CH>
__global__ void leaf_kernel(const int32_t *__restrict__ gptr, const int32_t *__restrict__ leaf_vtx,
                            const int32_t *__restrict__ leaf_dist, const int32_t *__restrict__ leaf_pdist,
                            const int32_t *__restrict__ leaf_lo, const int32_t *__restrict__ leaf_hi,
                            const T *__restrict__ F, int d, const float *__restrict__ ftab, float *__restrict__ leaf_out,
                            int max_gs) {
    extern __shared__ int smem_i[];
    const int gb = gptr[blockIdx.x], ge = gptr[blockIdx.x + 1], gs = ge - gb;
    const int c0 = blockIdx.y * CH;
    int levels = 1;
    while ((2 << (levels - 1)) <= max_gs) ++levels;
    int *sdist = smem_i;
    int *st = sdist + max_gs;                                   // levels x max_gs
    float *sx = reinterpret_cast<float *>(st + levels * max_gs);  // max_gs x CH
    for (int i = threadIdx.x; i < gs; i += blockDim.x) {
        sdist[i] = leaf_dist[gb + i];
        st[i] = leaf_pdist[gb + i];
        const int64_t v = leaf_vtx[gb + i];
#pragma unroll
        for (int c = 0; c < CH; ++c) sx[i * CH + c] = (c0 + c < d) ? to_f<T>(F[v * d + c0 + c]) : 0.f;
    }
    __syncthreads();
    for (int l = 1; (1 << l) <= gs; ++l) {
        const int h = 1 << (l - 1);
        for (int i = threadIdx.x; i + (1 << l) <= gs; i += blockDim.x)
            st[l * max_gs + i] = min(st[(l - 1) * max_gs + i], st[(l - 1) * max_gs + i + h]);
        __syncthreads();
    }
    for (int i = threadIdx.x; i < gs; i += blockDim.x) {
        const int lo = leaf_lo[gb + i] - gb, hi = leaf_hi[gb + i] - gb;
        const int di = sdist[i];
        float acc[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) acc[c] = 0.f;
        for (int j = lo; j < hi; ++j) {
            int dist = 0;
            if (j != i) {
                const int a = min(i, j) + 1, b = max(i, j);
                const int l = 31 - __clz(b - a + 1);
                const int m = min(st[l * max_gs + a], st[l * max_gs + b - (1 << l) + 1]);
                dist = di + sdist[j] - 2 * m;
            }
            const float f = __ldg(ftab + dist);
#pragma unroll
            for (int c = 0; c < CH; ++c) acc[c] = fmaf(f, sx[j * CH + c], acc[c]);
        }
        const int64_t v = leaf_vtx[gb + i];
#pragma unroll
        for (int c = 0; c < CH; ++c)
            if (c0 + c < d) leaf_out[v * d + c0 + c] = acc[c];
    }
}

}  // namespace dev
}  // namespace tfi
