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

// V consecutive field values of one row as FP32: one 16-byte (FP32) or 8-byte
// (BF16) load for V = 4; the caller guarantees the alignment.
template <typename T, int V>
__device__ __forceinline__ void load_row(const T *__restrict__ row, float *x) {
    if constexpr (V == 4 && sizeof(T) == 4) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(row));
        x[0] = q.x, x[1] = q.y, x[2] = q.z, x[3] = q.w;
    } else if constexpr (V == 4 && sizeof(T) == 2) {
        const uint2 q = __ldg(reinterpret_cast<const uint2 *>(row));
        const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162 *>(&q.x);
        const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162 *>(&q.y);
        x[0] = __low2float(a), x[1] = __high2float(a), x[2] = __low2float(b), x[3] = __high2float(b);
    } else {
#pragma unroll
        for (int i = 0; i < V; ++i) x[i] = to_f<T>(row[i]);
    }
}

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
        // up to four members at a time: all their index and row loads are in flight
        // together; the sum still runs in member order
        for (int e = key_ptr[k]; e < e1; e += 4) {
            int v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = e + q < e1 ? __ldg(key_vtx + e + q) : -1;
            float x[4][V];
#pragma unroll
            for (int q = 0; q < 4; ++q) load_row<T, V>(F + int64_t(v[q] < 0 ? v[0] : v[q]) * d + c, x[q]);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (v[q] < 0) break;
#pragma unroll
                for (int i = 0; i < V; ++i) acc[i] += x[q][i];
            }
        }
        float *dst = kbuf + k * d + c;
#pragma unroll
        for (int i = 0; i < V; ++i) dst[i] = acc[i];
    }
}

// ---------------------------------------------------------------------------
// bucket over segments: a bin's members are cut into consecutive segments of
// at most kBucketSeg members, so that a bin of a thousand vertices is summed
// by many threads instead of one. A segment that is its bin's only one writes
// the bin row (dst >= 0); the others write a partial row -1 - dst of sbuf,
// which bucket_combine adds up in segment order (a fixed order: deterministic).
// ---------------------------------------------------------------------------
template <typename T, int V>
__global__ void bucket_seg_kernel(int64_t n_segs, const int32_t *__restrict__ seg_ptr,
                                  const int32_t *__restrict__ seg_dst, const int32_t *__restrict__ key_vtx,
                                  const T *__restrict__ F, int d, float *__restrict__ kbuf, float *__restrict__ sbuf) {
    const int chunks = d / V;
    const int64_t total = n_segs * chunks;
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
        const int64_t g = t / chunks;
        const int c = int(t - g * chunks) * V;
        float acc[V];
#pragma unroll
        for (int i = 0; i < V; ++i) acc[i] = 0.f;
        const int e1 = seg_ptr[g + 1];
        for (int e = seg_ptr[g]; e < e1; e += 4) {
            int v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = e + q < e1 ? __ldg(key_vtx + e + q) : -1;
            float x[4][V];
#pragma unroll
            for (int q = 0; q < 4; ++q) load_row<T, V>(F + int64_t(v[q] < 0 ? v[0] : v[q]) * d + c, x[q]);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (v[q] < 0) break;
#pragma unroll
                for (int i = 0; i < V; ++i) acc[i] += x[q][i];
            }
        }
        const int dst = seg_dst[g];
        float *out = dst >= 0 ? kbuf + int64_t(dst) * d + c : sbuf + int64_t(-1 - dst) * d + c;
#pragma unroll
        for (int i = 0; i < V; ++i) out[i] = acc[i];
    }
}

// kbuf[mb_key[m]] = sum of the partial rows mb_ptr[m] .. mb_ptr[m + 1] - 1 of sbuf, in order
template <int V>
__global__ void bucket_combine(int64_t n_multi, const int32_t *__restrict__ mb_key, const int32_t *__restrict__ mb_ptr,
                               int d, const float *__restrict__ sbuf, float *__restrict__ kbuf) {
    const int chunks = d / V;
    const int64_t total = n_multi * chunks;
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
        const int64_t m = t / chunks;
        const int c = int(t - m * chunks) * V;
        float acc[V];
#pragma unroll
        for (int i = 0; i < V; ++i) acc[i] = 0.f;
        for (int r = mb_ptr[m]; r < mb_ptr[m + 1]; ++r) {
            float x[V];
            load_row<float, V>(sbuf + int64_t(r) * d + c, x);
#pragma unroll
            for (int i = 0; i < V; ++i) acc[i] += x[i];
        }
        float *out = kbuf + int64_t(mb_key[m]) * d + c;
#pragma unroll
        for (int i = 0; i < V; ++i) out[i] = acc[i];
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

// Shared-memory layout of one FFT array: element e lives at e + (e >> 5), one
// pad slot per 32 elements, so that the strided 8-byte accesses of the
// small-span passes spread over all banks.
__device__ __forceinline__ int padded(int e) { return e + (e >> 5); }
__host__ __device__ constexpr int padded_size(int np) { return np + (np >> 5); }

template <int RL>
__device__ __forceinline__ constexpr int brev_c(int q) {
    return RL == 1 ? q : RL == 2 ? (((q & 1) << 1) | (q >> 1)) : (((q & 1) << 2) | (q & 2) | ((q >> 2) & 1));
}

// Multiply by the constant twiddle exp(-2 pi i j / (2 dt)) (CONJ: its conjugate)
// for dt <= 4, without general complex products where the value is trivial.
template <int DT, int J, bool CONJ>
__device__ __forceinline__ float2 mul_c(float2 a) {
    constexpr float c = 0.70710678118654752f;
    if (J == 0) return a;
    if (DT == 2 || (DT == 4 && J == 2))  // -i (conjugate: +i)
        return CONJ ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
    if (J == 1)  // (1 - i)/sqrt2 (conjugate: (1 + i)/sqrt2)
        return CONJ ? make_float2(c * (a.x - a.y), c * (a.x + a.y)) : make_float2(c * (a.x + a.y), c * (a.y - a.x));
    // J == 3: (-1 - i)/sqrt2 (conjugate: (-1 + i)/sqrt2)
    return CONJ ? make_float2(-c * (a.x + a.y), c * (a.x - a.y)) : make_float2(c * (a.y - a.x), -c * (a.x + a.y));
}

// In-register 2^RL-point DFT, natural order in, bit-reversed order out (radix-2
// decimation in frequency with constant twiddles).
template <int RL>
__device__ __forceinline__ void dft_dif(float2 *v) {
    constexpr int R = 1 << RL;
#pragma unroll
    for (int st = RL - 1; st >= 0; --st) {
        const int dt = 1 << st;
#pragma unroll
        for (int t = 0; t < R; ++t) {
            if (t & dt) continue;
            const float2 a = v[t], b = v[t + dt];
            v[t] = make_float2(a.x + b.x, a.y + b.y);
            const float2 d = make_float2(a.x - b.x, a.y - b.y);
            const int j = t & (dt - 1);
            if (dt == 4) v[t + dt] = j == 0 ? d : j == 1 ? mul_c<4, 1, false>(d) : j == 2 ? mul_c<4, 2, false>(d) : mul_c<4, 3, false>(d);
            else if (dt == 2) v[t + dt] = j == 0 ? d : mul_c<2, 1, false>(d);
            else v[t + dt] = d;
        }
    }
}

// Inverse of dft_dif up to the factor 2^RL: bit-reversed in, natural out
// (radix-2 decimation in time with conjugate constant twiddles).
template <int RL>
__device__ __forceinline__ void idft_dit(float2 *v) {
    constexpr int R = 1 << RL;
#pragma unroll
    for (int st = 0; st < RL; ++st) {
        const int dt = 1 << st;
#pragma unroll
        for (int t = 0; t < R; ++t) {
            if (t & dt) continue;
            const int j = t & (dt - 1);
            const float2 b = v[t + dt];
            float2 x;
            if (dt == 4) x = j == 0 ? b : j == 1 ? mul_c<4, 1, true>(b) : j == 2 ? mul_c<4, 2, true>(b) : mul_c<4, 3, true>(b);
            else if (dt == 2) x = j == 0 ? b : mul_c<2, 1, true>(b);
            else x = b;
            const float2 a = v[t];
            v[t] = make_float2(a.x + x.x, a.y + x.y);
            v[t + dt] = make_float2(a.x - x.x, a.y - x.y);
        }
    }
}

// One radix-2^RL pass over RL consecutive radix-2 stages. Each thread takes
// groups of R = 2^RL elements of one axis at positions base + o + t h
// (h = 2^lh_lo, o < h, t < R), which are closed under the stages with
// half-spans h .. h R/2. Forward (decimation in frequency): an R-point DFT of
// the group, output k multiplied by w^k with w = exp(-2 pi i o / (R h)), stored
// at slot brev(k); this equals the RL radix-2 stages and keeps the overall
// natural -> bit-reversed order. INV is its exact inverse up to the factor R.
// The axis has length 2^ln and element stride es; 2^llog lines of stride ls;
// line_fast puts consecutive threads on consecutive lines.
template <bool INV, int RL>
__device__ __forceinline__ void fft_pass(float2 *Z, int padnp, int npair, int ln, int lh_lo, int es, int llog, int ls,
                                         bool line_fast, const float2 *__restrict__ tw) {
    constexpr int R = 1 << RL;
    const int glog = ln - RL;
    const int total = npair << (llog + glog);
    const int hmask = (1 << lh_lo) - 1;
    const int lmask = (1 << llog) - 1, gmask = (1 << glog) - 1;
    for (int w = threadIdx.x; w < total; w += blockDim.x) {
        int line, g;
        if (line_fast) {
            line = w & lmask;
            g = (w >> llog) & gmask;
        } else {
            g = w & gmask;
            line = (w >> glog) & lmask;
        }
        const int p = w >> (llog + glog);
        const int o = g & hmask;
        const int base = ((g >> lh_lo) << (lh_lo + RL)) + o;
        float2 *Zp = Z + p * padnp;
        // element t sits at e0 + t H; when H is a multiple of 32 the padding
        // grows by H / 32 per element, so its slot is padded(e0) + t (H + H / 32)
        const int e0 = line * ls + base * es, H = es << lh_lo;
        int adr[R];
        if ((H & 31) == 0) {
            const int a0 = padded(e0), st = H + (H >> 5);
#pragma unroll
            for (int t = 0; t < R; ++t) adr[t] = a0 + t * st;
        } else {
#pragma unroll
            for (int t = 0; t < R; ++t) adr[t] = padded(e0 + t * H);
        }
        float2 v[R];
#pragma unroll
        for (int t = 0; t < R; ++t) v[t] = Zp[adr[t]];
        // w^k with w = exp(-2 pi i o / (R h)), from the per-level entry
        // exp(-2 pi i o / (8 h)) by squaring
        float2 tws[R];
        if (lh_lo > 0) {
            const float2 w8 = __ldg(tw + (1 << lh_lo) + o);
            if (RL == 3) {
                tws[1] = w8;
                tws[2 % R] = cmul(w8, w8);
                tws[3 % R] = cmul(tws[1], tws[2 % R]);
                tws[4 % R] = cmul(tws[2 % R], tws[2 % R]);
                tws[5 % R] = cmul(tws[1], tws[4 % R]);
                tws[6 % R] = cmul(tws[2 % R], tws[4 % R]);
                tws[7 % R] = cmul(tws[3 % R], tws[4 % R]);
            } else if (RL == 2) {
                tws[1] = cmul(w8, w8);
                tws[2 % R] = cmul(tws[1], tws[1]);
                tws[3 % R] = cmul(tws[1], tws[2 % R]);
            } else {
                const float2 w4 = cmul(w8, w8);
                tws[1] = cmul(w4, w4);
            }
        }
        if (!INV) {
            dft_dif<RL>(v);
            if (lh_lo > 0) {
#pragma unroll
                for (int q = 1; q < R; ++q) v[q] = cmul(v[q], tws[brev_c<RL>(q)]);
            }
        } else {
            if (lh_lo > 0) {
#pragma unroll
                for (int q = 1; q < R; ++q) v[q] = cmulc(v[q], tws[brev_c<RL>(q)]);
            }
            idft_dit<RL>(v);
        }
#pragma unroll
        for (int t = 0; t < R; ++t) Zp[adr[t]] = v[t];
    }
    __syncthreads();
}

// All passes of one axis. Forward order runs from the largest span down: the
// 1- or 2-stage remainder pass first, then radix-8 passes ending at span 1;
// the inverse runs the mirror image. With skip_bottom the span-1 pass is left
// out (fused_bottom does it together with the spectrum product).
template <bool INV>
__device__ __forceinline__ void fft_axis(float2 *Z, int padnp, int npair, int ln, int es, int llog, int ls,
                                         bool line_fast, const float2 *__restrict__ tw, bool skip_bottom) {
    if (ln == 0) return;
    const int full = ln / 3, rem = ln - 3 * full;
    const bool do_rem = rem && !(skip_bottom && full == 0);
    if (!INV) {
        if (do_rem) {
            if (rem == 2) fft_pass<false, 2>(Z, padnp, npair, ln, ln - 2, es, llog, ls, line_fast, tw);
            else fft_pass<false, 1>(Z, padnp, npair, ln, ln - 1, es, llog, ls, line_fast, tw);
        }
        for (int k = 0; k < full; ++k) {
            const int lh = ln - rem - 3 * (k + 1);
            if (skip_bottom && lh == 0) break;
            fft_pass<false, 3>(Z, padnp, npair, ln, lh, es, llog, ls, line_fast, tw);
        }
    } else {
        for (int k = full - 1; k >= 0; --k) {
            const int lh = ln - rem - 3 * (k + 1);
            if (skip_bottom && lh == 0) continue;
            fft_pass<true, 3>(Z, padnp, npair, ln, lh, es, llog, ls, line_fast, tw);
        }
        if (do_rem) {
            if (rem == 2) fft_pass<true, 2>(Z, padnp, npair, ln, ln - 2, es, llog, ls, line_fast, tw);
            else fft_pass<true, 1>(Z, padnp, npair, ln, ln - 1, es, llog, ls, line_fast, tw);
        }
    }
}

// The span-1 pass of the innermost axis, forward and inverse, with the product
// by the kernel spectrum in between, all in registers (no twiddles at span 1).
template <int RL>
__device__ __forceinline__ void fused_bottom_pass(float2 *Z, int padnp, int npair, int ln, int es, int llog, int ls,
                                                  bool line_fast, const float2 *__restrict__ S, int s_pair) {
    constexpr int R = 1 << RL;
    const int glog = ln - RL;
    const int total = npair << (llog + glog);
    const int lmask = (1 << llog) - 1, gmask = (1 << glog) - 1;
    for (int w = threadIdx.x; w < total; w += blockDim.x) {
        int line, g;
        if (line_fast) {
            line = w & lmask;
            g = (w >> llog) & gmask;
        } else {
            g = w & gmask;
            line = (w >> glog) & lmask;
        }
        const int p = w >> (llog + glog);
        float2 *Zp = Z + p * padnp;
        const int e0 = line * ls + (g << RL) * es;
        int adr[R];
        if ((es & 31) == 0) {
            const int a0 = padded(e0), st = es + (es >> 5);
#pragma unroll
            for (int t = 0; t < R; ++t) adr[t] = a0 + t * st;
        } else {
#pragma unroll
            for (int t = 0; t < R; ++t) adr[t] = padded(e0 + t * es);
        }
        float2 sp[R], v[R];
        const float2 *Sp = S + p * s_pair;
#pragma unroll
        for (int q = 0; q < R; ++q) sp[q] = __ldg(Sp + e0 + q * es);
#pragma unroll
        for (int t = 0; t < R; ++t) v[t] = Zp[adr[t]];
        dft_dif<RL>(v);
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = cmul(v[q], sp[q]);
        idft_dit<RL>(v);
#pragma unroll
        for (int t = 0; t < R; ++t) Zp[adr[t]] = v[t];
    }
    __syncthreads();
}

// s_pair: offset between the spectra of consecutive arrays (0: one spectrum for all)
__device__ __forceinline__ void fused_bottom(float2 *Z, int padnp, int npair, int ln, int es, int llog, int ls,
                                             bool line_fast, const float2 *__restrict__ S, int s_pair = 0) {
    const int full = ln / 3, rem = ln - 3 * full;
    const int rl = full > 0 ? 3 : rem;
    if (rl == 3) fused_bottom_pass<3>(Z, padnp, npair, ln, es, llog, ls, line_fast, S, s_pair);
    else if (rl == 2) fused_bottom_pass<2>(Z, padnp, npair, ln, es, llog, ls, line_fast, S, s_pair);
    else fused_bottom_pass<1>(Z, padnp, npair, ln, es, llog, ls, line_fast, S, s_pair);
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
    const int padnp = padded_size(NP);
    const int npair = it.npair;
    {
        // 16-byte stores over the pairs of slots, then the odd last slot if any
        float4 *Z4 = reinterpret_cast<float4 *>(Z);
        const int nz = npair * padnp;
        for (int i = threadIdx.x; i < (nz >> 1); i += blockDim.x) Z4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if ((nz & 1) && threadIdx.x == 0) Z[nz - 1] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    const bool pair_io = (d & 1) == 0;   // channel pairs as one 8-byte access
    const int nk = jb.ke - jb.kb;
    // scatter bin sums; depth reversed so the depth correlation becomes a convolution
    for (int t = threadIdx.x; t < nk * npair; t += blockDim.x) {
        const int kk = t / npair, p = t - kk * npair;
        const int k = jb.kb + kk;
        const int ch = 2 * (it.pair0 + p);
        float re, im;
        if (pair_io) {
            const float2 q = __ldg(reinterpret_cast<const float2 *>(kbuf + int64_t(k) * d + ch));
            re = q.x, im = q.y;
        } else {
            re = kbuf[int64_t(k) * d + ch];
            im = (ch + 1 < d) ? kbuf[int64_t(k) * d + ch + 1] : 0.f;
        }
        const int pos = ((P1 - key_r[k]) & (P1 - 1)) * P2 + key_x[k];
        Z[p * padnp + padded(pos)] = make_float2(re, im);
    }
    __syncthreads();
    const float2 *S = spectra + jb.spec_off;
    if (lp1 > 0) {
        // rows (backbone axis) are the outer axis, columns (depth axis) the inner one
        fft_axis<false>(Z, padnp, npair, lp2, 1, lp1, P2, false, tw, false);
        fft_axis<false>(Z, padnp, npair, lp1, P2, lp2, 1, true, tw, true);
        fused_bottom(Z, padnp, npair, lp1, P2, lp2, 1, true, S);
        fft_axis<true>(Z, padnp, npair, lp1, P2, lp2, 1, true, tw, true);
        fft_axis<true>(Z, padnp, npair, lp2, 1, lp1, P2, false, tw, false);
    } else if (lp2 > 0) {
        fft_axis<false>(Z, padnp, npair, lp2, 1, 0, P2, false, tw, true);
        fused_bottom(Z, padnp, npair, lp2, 1, 0, P2, false, S);
        fft_axis<true>(Z, padnp, npair, lp2, 1, 0, P2, false, tw, true);
    } else {
        for (int p = threadIdx.x; p < npair; p += blockDim.x) Z[p * padnp] = cmul(Z[p * padnp], __ldg(S));
        __syncthreads();
    }
    for (int t = threadIdx.x; t < nk * npair; t += blockDim.x) {
        const int kk = t / npair, p = t - kk * npair;
        const int k = jb.kb + kk;
        const int ch = 2 * (it.pair0 + p);
        const float2 v = Z[p * padnp + padded(key_r[k] * P2 + key_x[k])];
        if (pair_io) {
            *reinterpret_cast<float2 *>(vbuf + int64_t(k) * d + ch) = v;
        } else {
            vbuf[int64_t(k) * d + ch] = v.x;
            if (ch + 1 < d) vbuf[int64_t(k) * d + ch + 1] = v.y;
        }
    }
}

// ---------------------------------------------------------------------------
// direct job kernel: one warp per (job, 64 query bins), two queries per lane,
// CH channels per pass; source bins staged through shared memory in chunks of
// 32 with a padded row stride so the row stores are conflict-free; the row
// updates run as paired FP32 FMAs (0.275 -> 0.238 ms per apply on the 2^20 tree)
// ---------------------------------------------------------------------------
// a0 += f x0 and a1 += f x1 as one packed two-lane FP32 FMA (each lane rounds
// like fmaf), halving the FMA instructions of the row updates
__device__ __forceinline__ void fma2(float &a0, float &a1, float f, float x0, float x1) {
    unsigned long long A, X, Fv;
    asm("mov.b64 %0, {%1, %2};" : "=l"(A) : "f"(a0), "f"(a1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(X) : "f"(x0), "f"(x1));
    asm("mov.b64 %0, {%1, %1};" : "=l"(Fv) : "f"(f));
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(A) : "l"(Fv), "l"(X));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a0), "=f"(a1) : "l"(A));
}

template <int CH>
struct SvStride {
    static constexpr int v = CH >= 8 ? CH + 4 : CH;
};

template <int CH, int WARPS, bool VEC>
__global__ void direct_kernel(const DirItem *__restrict__ items, int n_items, const JobDev *__restrict__ jobs,
                              const int32_t *__restrict__ key_r, const int32_t *__restrict__ key_x, int d,
                              const float *__restrict__ kbuf, float *__restrict__ vbuf, const float *__restrict__ ftab) {
    constexpr int SV = SvStride<CH>::v;
    __shared__ int sr[WARPS][32];
    __shared__ int sx[WARPS][32];
    __shared__ __align__(16) float sv[WARPS][32 * SV];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int w = blockIdx.x * WARPS + warp;
    if (w >= n_items) return;
    const int c0 = blockIdx.y * CH;
    const DirItem it = items[w];
    const JobDev jb = jobs[it.job];
    const int i0 = it.q0 + lane, i1 = i0 + 32;
    const bool v0 = i0 < jb.ke, v1 = i1 < jb.ke;
    const int r0 = v0 ? key_r[i0] : 0, x0 = v0 ? key_x[i0] : 0;
    const int r1 = v1 ? key_r[i1] : 0, x1 = v1 ? key_x[i1] : 0;
    float a0[CH], a1[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) a0[c] = a1[c] = 0.f;
    float *my = sv[warp];
    for (int s0 = jb.kb; s0 < jb.ke; s0 += 32) {
        const int j = s0 + lane;
        if (j < jb.ke) {
            sr[warp][lane] = key_r[j];
            sx[warp][lane] = key_x[j];
            const float *src = kbuf + int64_t(j) * d + c0;
            if (VEC) {
#pragma unroll
                for (int c = 0; c < CH; c += 4)
                    *reinterpret_cast<float4 *>(my + lane * SV + c) = *reinterpret_cast<const float4 *>(src + c);
            } else {
#pragma unroll
                for (int c = 0; c < CH; ++c) my[lane * SV + c] = (c0 + c < d) ? src[c] : 0.f;
            }
        }
        __syncwarp();
        const int cnt = min(32, jb.ke - s0);
        for (int t = 0; t < cnt; ++t) {
            const int rt = sr[warp][t], xt = sx[warp][t];
            const float f0 = __ldg(ftab + r0 + rt + abs(x0 - xt));
            const float f1 = __ldg(ftab + r1 + rt + abs(x1 - xt));
            if (VEC) {
#pragma unroll
                for (int c = 0; c < CH; c += 4) {
                    const float4 q = *reinterpret_cast<const float4 *>(my + t * SV + c);
                    fma2(a0[c], a0[c + 1], f0, q.x, q.y);
                    fma2(a0[c + 2], a0[c + 3], f0, q.z, q.w);
                    fma2(a1[c], a1[c + 1], f1, q.x, q.y);
                    fma2(a1[c + 2], a1[c + 3], f1, q.z, q.w);
                }
            } else {
#pragma unroll
                for (int c = 0; c < CH; ++c) {
                    const float q = my[t * SV + c];
                    a0[c] = fmaf(f0, q, a0[c]);
                    a1[c] = fmaf(f1, q, a1[c]);
                }
            }
        }
        __syncwarp();
    }
    if (VEC) {
        if (v0) {
#pragma unroll
            for (int c = 0; c < CH; c += 4)
                *reinterpret_cast<float4 *>(vbuf + int64_t(i0) * d + c0 + c) = make_float4(a0[c], a0[c + 1], a0[c + 2], a0[c + 3]);
        }
        if (v1) {
#pragma unroll
            for (int c = 0; c < CH; c += 4)
                *reinterpret_cast<float4 *>(vbuf + int64_t(i1) * d + c0 + c) = make_float4(a1[c], a1[c + 1], a1[c + 2], a1[c + 3]);
        }
    } else {
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            if (c0 + c < d) {
                if (v0) vbuf[int64_t(i0) * d + c0 + c] = a0[c];
                if (v1) vbuf[int64_t(i1) * d + c0 + c] = a1[c];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// gather: out[u] = leaf[u] + sum_calls (val[A-bin] - val[b-bin]), vertices taken
// in a depth-first order of the tree; rec_ptr, akey, bkey, the leaf rows and
// in_leaf are indexed by that order's positions (u = order[i] has records
// rec_ptr[i] .. rec_ptr[i + 1] - 1 and its leaf term in row i)
// ---------------------------------------------------------------------------
template <typename T, int V>
__global__ void gather_kernel(int n, const int32_t *__restrict__ order, const int32_t *__restrict__ rec_ptr,
                              const int32_t *__restrict__ akey, const int32_t *__restrict__ bkey,
                              const float *__restrict__ vbuf, const float *__restrict__ leaf,
                              const uint8_t *__restrict__ in_leaf, int d, T *__restrict__ out) {
    const int chunks = d / V;
    const int64_t total = int64_t(n) * chunks;
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
        const int64_t i = t / chunks;
        const int c = int(t - i * chunks) * V;
        // vertices in depth-first order: neighbouring threads share most of their
        // calls' table rows, which then come from L2 rather than DRAM
        const int64_t u = order[i];
        float acc[V];
        if (in_leaf[i] != 0) {
            load_row<float, V>(leaf + i * d + c, acc);
        } else {
#pragma unroll
            for (int i = 0; i < V; ++i) acc[i] = 0.f;
        }
        const int e1 = rec_ptr[i + 1];
        // up to four records at a time: their key and row loads are in flight together;
        // the sum still runs in record order
        for (int e = rec_ptr[i]; e < e1; e += 4) {
            int ka[4], kb[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const bool ok = e + q < e1;
                ka[q] = ok ? __ldg(akey + e + q) : -1;
                kb[q] = ok ? __ldg(bkey + e + q) : -1;
            }
            float g[4][V], h[4][V];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                load_row<float, V>(vbuf + int64_t(ka[q] < 0 ? ka[0] : ka[q]) * d + c, g[q]);
                if (kb[q] >= 0) {
                    load_row<float, V>(vbuf + int64_t(kb[q]) * d + c, h[q]);
                } else {
#pragma unroll
                    for (int i = 0; i < V; ++i) h[q][i] = 0.f;
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (ka[q] < 0) break;
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    acc[i] += g[q][i];
                    if (kb[q] >= 0) acc[i] -= h[q][i];
                }
            }
        }
        T *dst = out + u * d + c;
        if constexpr (V == 4 && sizeof(T) == 4) {
            *reinterpret_cast<float4 *>(dst) = make_float4(acc[0], acc[1], acc[2], acc[3]);
        } else {
#pragma unroll
            for (int i = 0; i < V; ++i) dst[i] = from_f<T>(acc[i]);
        }
    }
}

// ---------------------------------------------------------------------------
// dense leaves of fewer than kLeafWarpMin vertices: one CTA per group of
// consecutive small leaves, CH channels per pass.
// In a leaf's preorder, dhat(i, j) = D(i) + D(j) - 2 min_{w in (min(i,j), max(i,j)]}
// D(parent(w)). Each target i walks all sources of its leaf in one order with a
// running minimum: first j = i+1 .. hi-1 (min over (i, j] grows by one entry),
// then j = hi-2-k downwards over j < i (min over (j, i]). In the first phase
// neighbouring threads read neighbouring rows; in the second every thread of a
// leaf reads the same row. Field rows use a padded stride, and the f samples are
// staged in shared memory when they fit.
// ---------------------------------------------------------------------------
template <int CH>
struct LeafStride {
    static constexpr int v = CH >= 8 ? CH + 4 : CH;
};

__host__ __device__ inline size_t leaf_smem_bytes(int max_gs, int ch, int ftab_smem) {
    const int sv = ch >= 8 ? ch + 4 : ch;
    return size_t(2 * max_gs + 4) * 4 + size_t(max_gs) * sv * 4 + size_t(ftab_smem) * 4;
}

// FS: the f samples are staged in shared memory (ftab_smem > 0). As a template
// argument it lets the compiler emit shared-memory loads for the f lookups; a
// pointer chosen at run time between shared and global memory makes them
// generic loads.
template <typename T, int CH, bool FS>
__global__ void leaf_kernel(const int32_t *__restrict__ gptr, const int32_t *__restrict__ leaf_vtx,
                            const int32_t *__restrict__ leaf_dist, const int32_t *__restrict__ leaf_pdist,
                            const int32_t *__restrict__ leaf_lo, const int32_t *__restrict__ leaf_hi,
                            const T *__restrict__ F, int d, const float *__restrict__ ftab, int ftab_smem,
                            float *__restrict__ leaf_out, const int32_t *__restrict__ leaf_row, int max_gs) {
    constexpr int SV = LeafStride<CH>::v;
    extern __shared__ __align__(16) int smem_i[];
    const int gb = gptr[2 * blockIdx.x], ge = gptr[2 * blockIdx.x + 1], gs = ge - gb;  // [begin, end) pairs
    const int c0 = blockIdx.y * CH;
    int *sdist = smem_i;
    int *spd = sdist + max_gs;
    float *sx = reinterpret_cast<float *>(smem_i + ((2 * max_gs + 3) & ~3));   // 16-byte aligned rows
    float *sf = sx + max_gs * SV;
    for (int i = threadIdx.x; i < gs; i += blockDim.x) {
        sdist[i] = leaf_dist[gb + i];
        spd[i] = leaf_pdist[gb + i];
        const int64_t v = leaf_vtx[gb + i];
#pragma unroll
        for (int c = 0; c < CH; ++c) sx[i * SV + c] = (c0 + c < d) ? to_f<T>(F[v * d + c0 + c]) : 0.f;
    }
    for (int i = threadIdx.x; i < ftab_smem; i += blockDim.x) sf[i] = ftab[i];
    __syncthreads();
    const float *fsrc = FS ? sf : ftab;
    for (int i = threadIdx.x; i < gs; i += blockDim.x) {
        const int lo = leaf_lo[gb + i] - gb, hi = leaf_hi[gb + i] - gb;
        const int di = sdist[i];
        float acc[CH];
        const float f0 = fsrc[0];
#pragma unroll
        for (int c = 0; c < CH; ++c) acc[c] = f0 * sx[i * SV + c];
        const int nf = hi - 1 - i;              // sources after i
        const int steps = hi - lo - 1;          // all sources but i
        int m = 0x7fffffff;
        for (int k = 0; k < steps; ++k) {
            int j;
            if (k < nf) {
                j = i + 1 + k;
                m = min(m, spd[j]);
            } else {
                if (k == nf) m = 0x7fffffff;
                j = hi - 2 - k;
                m = min(m, spd[j + 1]);
            }
            const float f = fsrc[di + sdist[j] - 2 * m];
            if (CH % 4 == 0) {
#pragma unroll
                for (int c = 0; c < CH; c += 4) {
                    const float4 q = *reinterpret_cast<const float4 *>(sx + j * SV + c);
                    acc[c] = fmaf(f, q.x, acc[c]);
                    acc[c + 1] = fmaf(f, q.y, acc[c + 1]);
                    acc[c + 2] = fmaf(f, q.z, acc[c + 2]);
                    acc[c + 3] = fmaf(f, q.w, acc[c + 3]);
                }
            } else {
#pragma unroll
                for (int c = 0; c < CH; ++c) acc[c] = fmaf(f, sx[j * SV + c], acc[c]);
            }
        }
        const int64_t v = leaf_row[gb + i];
#pragma unroll
        for (int c = 0; c < CH; ++c)
            if (c0 + c < d) leaf_out[v * d + c0 + c] = acc[c];
    }
}

// ---------------------------------------------------------------------------
// dense leaves of at least kLeafWarpMin vertices: CTAs of eight warps, each
// running one or more big leaves packed on the host (a leaf takes ceil(size / 64)
// warps, all eight when it is alone; the CTA stages its leaves one after
// another), one warp per block of 32 kLeafWarpTargets consecutive targets, each
// lane holding the targets a + lane + 32k (k < kLeafWarpTargets). Packing keeps
// every warp busy where one CTA per leaf left the warps of a leaf below 512
// vertices idle. Registers are capped for three CTAs per SM. All lanes
// visit the same source at the same time, so every field-row and
// parent-distance load is a shared-memory broadcast, and each row a lane loads
// feeds all its targets (shared memory delivers 128 bytes per cycle to the
// lanes whatever the addresses, so the reuse in registers is what lifts the
// kernel off that limit; two targets per lane measured faster than one or four,
// which cost occupancy and masked work on the block diagonal). With the block
// [a, e):
//   sources after the block, ascending: m_i = min(m_i, pd[j]) from
//     m_i = min pd over (i, e - 1] (chunked warp suffix minima);
//   sources before the block, descending: m_i = min(m_i, pd[j + 1]) from
//     m_i = min pd over (a, i] (chunked warp prefix minima);
//   sources inside the block: one ascending sweep for j > i and one descending
//   sweep for j < i, each starting from an empty minimum.
// ---------------------------------------------------------------------------
constexpr int kLeafWarpMin = 64;
constexpr int kLeafWarpTargets = 2;  // targets per lane in leaf_warp_kernel (a warp covers 64)

// source rows are only read as broadcasts here, so they need no padding (stride CH)
__host__ __device__ inline size_t leaf_warp_smem_bytes(int max_leaf, int ch, int ftab_smem) {
    return size_t(2 * max_leaf + 4) * 4 + size_t(max_leaf) * ch * 4 + size_t(ftab_smem) * 4;
}

template <typename T, int CH, bool FS>  // FS as in leaf_kernel
__global__ void __launch_bounds__(256, 3) leaf_warp_kernel(const int32_t *__restrict__ big_ptr,
                                                           const int32_t *__restrict__ big_lo,
                                                           const int32_t *__restrict__ big_hi,
                                                           const int32_t *__restrict__ leaf_vtx,
                                                           const int32_t *__restrict__ leaf_dist,
                                                           const int32_t *__restrict__ leaf_pdist, const T *__restrict__ F,
                                                           int d, const float *__restrict__ ftab, int ftab_smem,
                                                           float *__restrict__ leaf_out,
                                                           const int32_t *__restrict__ leaf_row, int max_leaf) {
    constexpr int SV = CH;
    constexpr int INF = 0x7fffffff;
    constexpr int TT = kLeafWarpTargets;  // targets per lane, 32 apart
    constexpr int BLK = 32 * TT;          // targets of one warp
    extern __shared__ __align__(16) int smem_i[];
    // the CTA's leaves big_lo/hi[q0 .. q1), staged one after another (at most max_leaf vertices)
    const int q0 = big_ptr[blockIdx.x], q1 = big_ptr[blockIdx.x + 1];
    const int c0 = blockIdx.y * CH;
    int *sdist = smem_i;
    int *spd = sdist + max_leaf;
    float *sx = reinterpret_cast<float *>(smem_i + ((2 * max_leaf + 3) & ~3));
    float *sf = sx + max_leaf * SV;
    for (int q = q0, off = 0; q < q1; ++q) {
        const int lo = big_lo[q], n = big_hi[q] - lo;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            sdist[off + i] = leaf_dist[lo + i];
            spd[off + i] = leaf_pdist[lo + i];
            const int64_t v = leaf_vtx[lo + i];
#pragma unroll
            for (int c = 0; c < CH; ++c) sx[(off + i) * SV + c] = (c0 + c < d) ? to_f<T>(F[v * d + c0 + c]) : 0.f;
        }
        off += n;
    }
    for (int i = threadIdx.x; i < ftab_smem; i += blockDim.x) sf[i] = ftab[i];
    __syncthreads();
    const float *fsrc = FS ? sf : ftab;
    // this warp's leaf: the leaves take consecutive warps, ceil(size / BLK) each, or all
    // warps when a leaf is alone; warps past the last leaf have nothing to do
    const int lane = threadIdx.x & 31, cw = threadIdx.x >> 5, cwarps = blockDim.x >> 5;
    int lb = 0, ls = 0, warp = -1, nwarps = 1, off = 0;
    for (int q = q0, w0 = 0, o = 0; q < q1; ++q) {
        const int n = big_hi[q] - big_lo[q];
        const int W = q1 - q0 == 1 ? cwarps : min(cwarps - w0, (n + BLK - 1) / BLK);
        if (cw >= w0 && cw < w0 + W) {
            lb = big_lo[q];
            ls = n;
            warp = cw - w0;
            nwarps = W;
            off = o;
        }
        w0 += W;
        o += n;
    }
    if (warp < 0) return;  // no block-wide barrier follows
    sdist += off;
    spd += off;
    sx += off * SV;
    for (int a = warp * BLK; a < ls; a += nwarps * BLK) {
        const int bend = min(a + BLK, ls);  // the warp's targets are [a, bend)
        int ti[TT], D[TT], m[TT];
        bool act[TT];
        float acc[TT][CH];
#pragma unroll
        for (int k = 0; k < TT; ++k) {
            ti[k] = a + 32 * k + lane;
            act[k] = ti[k] < ls;
            D[k] = act[k] ? sdist[ti[k]] : 0;
#pragma unroll
            for (int c = 0; c < CH; ++c) acc[k][c] = 0.f;
        }
        // one source row for all targets of the lane: f[k] x row
        auto add = [&](const float *f, int j) {
            const float *x = sx + j * SV;
            if (CH % 4 == 0) {
#pragma unroll
                for (int c = 0; c < CH; c += 4) {
                    const float4 q = *reinterpret_cast<const float4 *>(x + c);
#pragma unroll
                    for (int k = 0; k < TT; ++k) {
                        fma2(acc[k][c], acc[k][c + 1], f[k], q.x, q.y);
                        fma2(acc[k][c + 2], acc[k][c + 3], f[k], q.z, q.w);
                    }
                }
            } else {
#pragma unroll
                for (int c = 0; c < CH; ++c) {
                    const float q = x[c];
#pragma unroll
                    for (int k = 0; k < TT; ++k) acc[k][c] = fmaf(f[k], q, acc[k][c]);
                }
            }
        };
        // sources inside the block: j > i ascending, then j < i descending
#pragma unroll
        for (int k = 0; k < TT; ++k) m[k] = INF;
        for (int j = a; j < bend; ++j) {
            const int p = spd[j], dj = sdist[j];
            float f[TT];
#pragma unroll
            for (int k = 0; k < TT; ++k) {
                if (j > ti[k]) m[k] = min(m[k], p);
                f[k] = !act[k] ? 0.f : j == ti[k] ? fsrc[0] : j > ti[k] ? fsrc[D[k] + dj - 2 * m[k]] : 0.f;
            }
            add(f, j);
        }
#pragma unroll
        for (int k = 0; k < TT; ++k) m[k] = INF;
        for (int j = bend - 1; j >= a; --j) {
            const int p = spd[j + 1 < ls ? j + 1 : j], dj = sdist[j];
            float f[TT];
#pragma unroll
            for (int k = 0; k < TT; ++k) {
                if (j < ti[k]) m[k] = min(m[k], p);
                f[k] = (act[k] && j < ti[k]) ? fsrc[D[k] + dj - 2 * m[k]] : 0.f;
            }
            add(f, j);
        }
        // carries at the block edges from chunked warp scans of the block's parent
        // distances P[t] = pd[a + t]: suffix min over (i, bend - 1], prefix min over (a, i]
        int suf[TT], pre[TT];
        {
            int cmin[TT], cpre[TT];
#pragma unroll
            for (int k = 0; k < TT; ++k) {
                const int t = 32 * k + lane;
                // suffix within chunk k over elements t + 1 .. 32k + 31
                int v = (a + t + 1 < bend && lane < 31) ? spd[a + t + 1] : INF;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int u = __shfl_down_sync(0xffffffffu, v, o);
                    if (lane + o < 32) v = min(v, u);
                }
                suf[k] = v;
                // prefix within chunk k over elements 32k .. t, element 0 excluded
                int w = (a + t < bend && t > 0) ? spd[a + t] : INF;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int u = __shfl_up_sync(0xffffffffu, w, o);
                    if (lane >= o) w = min(w, u);
                }
                pre[k] = w;
                cpre[k] = __shfl_sync(0xffffffffu, w, 31);   // min over the whole chunk (element 0 excluded)
                const int e = (a + t < bend) ? spd[a + t] : INF;
                int cm = e;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) cm = min(cm, __shfl_xor_sync(0xffffffffu, cm, o));
                cmin[k] = cm;                                 // min over all of chunk k
            }
            // combine chunks: suffix adds the chunks after k (their first element
            // included), prefix adds the chunks before k
            int after = INF;
#pragma unroll
            for (int k = TT - 1; k >= 0; --k) {
                suf[k] = min(suf[k], after);
                after = min(after, cmin[k]);
            }
            int before = INF;
#pragma unroll
            for (int k = 0; k < TT; ++k) {
                pre[k] = min(pre[k], before);
                before = min(before, cpre[k]);
            }
        }
        // sources after the block
        constexpr int U = 2;  // sources per step (four spill at the 80-register cap)
#pragma unroll
        for (int k = 0; k < TT; ++k) m[k] = suf[k];
        int j = bend;
        for (; j + U <= ls; j += U) {
            float f[U][TT];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int p = spd[j + u], dj = sdist[j + u];
#pragma unroll
                for (int k = 0; k < TT; ++k) {
                    m[k] = min(m[k], p);
                    f[u][k] = act[k] ? fsrc[D[k] + dj - 2 * m[k]] : 0.f;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) add(f[u], j + u);
        }
        for (; j < ls; ++j) {
            const int p = spd[j], dj = sdist[j];
            float f[TT];
#pragma unroll
            for (int k = 0; k < TT; ++k) {
                m[k] = min(m[k], p);
                f[k] = act[k] ? fsrc[D[k] + dj - 2 * m[k]] : 0.f;
            }
            add(f, j);
        }
        // sources before the block
#pragma unroll
        for (int k = 0; k < TT; ++k) m[k] = pre[k];
        j = a - 1;
        for (; j - U + 1 >= 0; j -= U) {
            float f[U][TT];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int p = spd[j - u + 1], dj = sdist[j - u];
#pragma unroll
                for (int k = 0; k < TT; ++k) {
                    m[k] = min(m[k], p);
                    f[u][k] = act[k] ? fsrc[D[k] + dj - 2 * m[k]] : 0.f;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) add(f[u], j - u);
        }
        for (; j >= 0; --j) {
            const int p = spd[j + 1], dj = sdist[j];
            float f[TT];
#pragma unroll
            for (int k = 0; k < TT; ++k) {
                m[k] = min(m[k], p);
                f[k] = act[k] ? fsrc[D[k] + dj - 2 * m[k]] : 0.f;
            }
            add(f, j);
        }
#pragma unroll
        for (int k = 0; k < TT; ++k) {
            if (act[k]) {
                float *dst = leaf_out + int64_t(leaf_row[lb + ti[k]]) * d;
#pragma unroll
                for (int c = 0; c < CH; ++c)
                    if (c0 + c < d) dst[c0 + c] = acc[k][c];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Exponential-sum sweeps (Algorithm 7, "CrossSubRoutineExp") for kernels
// f(k delta) = sum_l c_l exp(-beta_l k), beta_l = b_l delta per grid unit.
// For one term, G_q[s] = lambda^q G_0[s] and E_alpha[q] = lambda^q E_alpha[0]
// (Eq. "stad-specialized-factorization"), so every bin value the gather reads
// is c lambda^r times G_0 at its backbone vertex (A-bins) or E_alpha[0] (b-bins).
// G_0[t] = sum_s lambda^{|X_t - X_s|} a_s with a_s = sum over the vertices
// projecting to p_s of lambda^{d(v)} x_v, computed as a forward partial sum
// Fw[t] = a_t + lambda^{X_t - X_{t-1}} Fw[t-1], a backward one Bw likewise, and
// G_0 = Fw + Bw - a (the paper's backward update (1 - lambda^2) G + lambda G
// rewritten as two positive recurrences; the same value in exact arithmetic).
// ---------------------------------------------------------------------------
struct SweepJobDev {
    int32_t sb, se, rb, m, cjb, cje;
};

// One warp per job and block of kSweepCH channels (blockIdx.y). Run sums are
// reductions over keys: lanes take keys 32 apart, each accumulating the whole
// channel block (lambda^r computed once per key and term), then a butterfly of
// shuffles (fixed order: deterministic) leaves every lane with the totals; the
// recurrences over the backbone runs are evaluated redundantly by all lanes.
constexpr int kSweepCH = 16;

__device__ __forceinline__ void sweep_row_acc(float *acc, const float *__restrict__ row, int nch, bool vec4, float w) {
    if (vec4) {
#pragma unroll
        for (int c = 0; c < kSweepCH; c += 4) {
            if (c < nch) {
                const float4 q = __ldg(reinterpret_cast<const float4 *>(row + c));
                acc[c] = fmaf(w, q.x, acc[c]);
                acc[c + 1] = fmaf(w, q.y, acc[c + 1]);
                acc[c + 2] = fmaf(w, q.z, acc[c + 2]);
                acc[c + 3] = fmaf(w, q.w, acc[c + 3]);
            }
        }
    } else {
#pragma unroll
        for (int c = 0; c < kSweepCH; ++c)
            if (c < nch) acc[c] = fmaf(w, __ldg(row + c), acc[c]);
    }
}

__device__ __forceinline__ void sweep_warp_sum(float *acc) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int c = 0; c < kSweepCH; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
    }
}

// row[c] (+)= w * g[c] for the channel block
__device__ __forceinline__ void sweep_row_out(float *__restrict__ row, const float *g, int nch, float w, bool first) {
#pragma unroll
    for (int c = 0; c < kSweepCH; ++c)
        if (c < nch) row[c] = first ? w * g[c] : row[c] + w * g[c];
}

template <int WARPS>
__global__ void sweep_g_kernel(const SweepJobDev *__restrict__ jobs, int n_jobs, const int32_t *__restrict__ key_r,
                               const int32_t *__restrict__ key_x, const int32_t *__restrict__ sw_keys,
                               const int32_t *__restrict__ sw_run, int d, const float *__restrict__ kbuf,
                               float *__restrict__ vbuf, float *__restrict__ scratch, const float *__restrict__ beta,
                               const float *__restrict__ coef, int J) {
    const int w = blockIdx.x * WARPS + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (w >= n_jobs) return;
    const SweepJobDev jb = jobs[w];
    const int c0 = blockIdx.y * kSweepCH, nch = min(kSweepCH, d - c0);
    const bool vec4 = (d % 4) == 0;
    for (int l = 0; l < J; ++l) {
        const float b = beta[l], cl = coef[l];
        float fw[kSweepCH];
        int prev_x = 0;
        for (int t = 0; t < jb.m; ++t) {
            const int e0 = sw_run[jb.rb + t], e1 = sw_run[jb.rb + t + 1];
            const int x = key_x[sw_keys[e0]];
            float a[kSweepCH];
#pragma unroll
            for (int c = 0; c < kSweepCH; ++c) a[c] = 0.f;
            for (int e = e0 + lane; e < e1; e += 32) {
                const int k = sw_keys[e];
                sweep_row_acc(a, kbuf + int64_t(k) * d + c0, nch, vec4, expf(-b * float(key_r[k])));
            }
            sweep_warp_sum(a);
            const float dec = t == 0 ? 0.f : expf(-b * float(x - prev_x));
#pragma unroll
            for (int c = 0; c < kSweepCH; ++c) fw[c] = t == 0 ? a[c] : a[c] + dec * fw[c];
            // lane c keeps channel c of (Fw, a) for the backward sweep
            if (lane < nch) {
                float fv = 0.f, av = 0.f;
#pragma unroll
                for (int c = 0; c < kSweepCH; ++c)
                    if (c == lane) fv = fw[c], av = a[c];
                scratch[(int64_t(jb.rb + t) * 2) * d + c0 + lane] = fv;
                scratch[(int64_t(jb.rb + t) * 2 + 1) * d + c0 + lane] = av;
            }
            prev_x = x;
        }
        __syncwarp();
        float bw[kSweepCH];
        int next_x = 0;
        for (int t = jb.m - 1; t >= 0; --t) {
            const int e0 = sw_run[jb.rb + t], e1 = sw_run[jb.rb + t + 1];
            const int x = key_x[sw_keys[e0]];
            const float dec = t == jb.m - 1 ? 0.f : expf(-b * float(next_x - x));
            float g0[kSweepCH];
#pragma unroll
            for (int c = 0; c < kSweepCH; ++c) {
                const float av = c < nch ? scratch[(int64_t(jb.rb + t) * 2 + 1) * d + c0 + c] : 0.f;
                const float fv = c < nch ? scratch[(int64_t(jb.rb + t) * 2) * d + c0 + c] : 0.f;
                bw[c] = t == jb.m - 1 ? av : av + dec * bw[c];
                g0[c] = fv + bw[c] - av;   // G_0 = Fw + Bw - a (a_s counted by both sweeps)
            }
            for (int e = e0 + lane; e < e1; e += 32) {
                const int k = sw_keys[e];
                sweep_row_out(vbuf + int64_t(k) * d + c0, g0, nch, cl * expf(-b * float(key_r[k])), l == 0);
            }
            next_x = x;
        }
        __syncwarp();
    }
}

template <int WARPS>
__global__ void sweep_e_kernel(const int32_t *__restrict__ ejobs, int n_jobs, const JobDev *__restrict__ jobs,
                               const int32_t *__restrict__ key_r, int d, const float *__restrict__ kbuf,
                               float *__restrict__ vbuf, const float *__restrict__ beta,
                               const float *__restrict__ coef, int J) {
    const int w = blockIdx.x * WARPS + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (w >= n_jobs) return;
    const JobDev jb = jobs[ejobs[w]];
    const int c0 = blockIdx.y * kSweepCH, nch = min(kSweepCH, d - c0);
    const bool vec4 = (d % 4) == 0;
    for (int l = 0; l < J; ++l) {
        const float b = beta[l], cl = coef[l];
        float e0v[kSweepCH];   // E_alpha[0] = sum_r lambda^r b_alpha[r]
#pragma unroll
        for (int c = 0; c < kSweepCH; ++c) e0v[c] = 0.f;
        for (int k = jb.kb + lane; k < jb.ke; k += 32)
            sweep_row_acc(e0v, kbuf + int64_t(k) * d + c0, nch, vec4, expf(-b * float(key_r[k])));
        sweep_warp_sum(e0v);
        for (int k = jb.kb + lane; k < jb.ke; k += 32)
            sweep_row_out(vbuf + int64_t(k) * d + c0, e0v, nch, cl * expf(-b * float(key_r[k])), l == 0);
    }
}

// ---------------------------------------------------------------------------
// Sinkhorn scaling update (Eq. "app-sinkhorn-updates"): out = marg / (Kx + delta)
// ---------------------------------------------------------------------------
__global__ void sinkhorn_scale(int64_t n, const float *__restrict__ marg, const float *__restrict__ Kx, float delta,
                               float *__restrict__ out) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        out[i] = marg[i] / (Kx[i] + delta);
}

// Table values of the bins a support truncation left out of their tables: zero rows
// [ranges[2i], ranges[2i + 1]) of vbuf, one CTA row per range.
__global__ void zero_rows(const int32_t *__restrict__ ranges, int n_ranges, int d, float *__restrict__ vbuf) {
    for (int r = blockIdx.y; r < n_ranges; r += gridDim.y) {
        const int64_t b = int64_t(ranges[2 * r]) * d, e = int64_t(ranges[2 * r + 1]) * d;
        for (int64_t i = b + blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < e; i += int64_t(gridDim.x) * blockDim.x)
            vbuf[i] = 0.f;
    }
}

__global__ void fill_value(int64_t n, float v, float *__restrict__ out) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        out[i] = v;
}

// ---------------------------------------------------------------------------
// (a2) distances and bin keys on the device, at plan time.
// Root grid distances D and hop depths by pointer doubling over the rooted
// parent array (a prefix sum along every root path: D_{k+1}[v] = D_k[v] +
// D_k[J_k[v]], J_{k+1} = J_k o J_k, with D = 0 and J = itself at a root); the
// jump tables J_k double as binary-lifting ancestor tables for the LCA. Then per
// record (v in call S, anchor a = pi(v), backbone start p_1):
//   d(v)     = D(v)   + D(a) - 2 D(lca(v, a))      (Eq. "stad-depth")
//   X(pi v)  = D(p_1) + D(a) - 2 D(lca(p_1, a))    (backbone coordinate)
// ---------------------------------------------------------------------------
__global__ void k1_init(int n, const int32_t *__restrict__ parent, const int32_t *__restrict__ qpar,
                        int64_t *__restrict__ D, int32_t *__restrict__ hop, int32_t *__restrict__ anc0) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int p = parent[v];
        anc0[v] = p;
        D[v] = p == v ? 0 : qpar[v];
        hop[v] = p == v ? 0 : 1;
    }
}

__global__ void k1_jump(int n, const int32_t *__restrict__ anc_k, const int64_t *__restrict__ Din,
                        const int32_t *__restrict__ hin, int32_t *__restrict__ anc_k1, int64_t *__restrict__ Dout,
                        int32_t *__restrict__ hout) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int a = anc_k[v];
        anc_k1[v] = anc_k[a];
        Dout[v] = Din[v] + Din[a];
        hout[v] = hin[v] + hin[a];
    }
}

__device__ __forceinline__ int k1_lca(int u, int v, const int32_t *__restrict__ anc, int n, int K,
                                      const int32_t *__restrict__ hop) {
    if (hop[u] < hop[v]) {
        const int t = u;
        u = v;
        v = t;
    }
    int diff = hop[u] - hop[v];
    for (int k = 0; diff; ++k, diff >>= 1)
        if (diff & 1) u = anc[int64_t(k) * n + u];
    if (u == v) return u;
    for (int k = K - 1; k >= 0; --k) {
        const int au = anc[int64_t(k) * n + u], av = anc[int64_t(k) * n + v];
        if (au != av) {
            u = au;
            v = av;
        }
    }
    return anc[u];
}

__global__ void k1_records(int64_t R, const int32_t *__restrict__ rec_v, const int32_t *__restrict__ rec_a,
                           const int32_t *__restrict__ rec_p1, const int64_t *__restrict__ D,
                           const int32_t *__restrict__ hop, const int32_t *__restrict__ anc, int n, int K,
                           int32_t *__restrict__ out_r, int32_t *__restrict__ out_x) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < R; i += int64_t(gridDim.x) * blockDim.x) {
        const int v = rec_v[i], a = rec_a[i], p1 = rec_p1[i];
        out_r[i] = int32_t(D[v] + D[a] - 2 * D[k1_lca(v, a, anc, n, K, hop)]);
        out_x[i] = int32_t(D[p1] + D[a] - 2 * D[k1_lca(p1, a, anc, n, K, hop)]);
    }
}

}  // namespace dev
}  // namespace tfi
