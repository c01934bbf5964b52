// Cross tables and corrections too large for one CTA's shared memory (P = P1 P2
// grid points with P > 2^14): the circular correlation of Eq.
// "stad-2d-convolution" (Eq. "stad-E" for a correction) evaluated by a four-step
// FFT through a global-memory buffer, one P-point complex array per (table,
// channel pair).
//
// The outer (depth) axis of length P1 = N1a N1b is split into a column index na
// and a block-row index nb: grid point (n1, x) with n1 = na N1b + nb lives at
// na BLK + nb P2 + x, BLK = N1b P2. With the outer frequency k1 = ka + N1a kb,
//   X[k1, kx] = sum_{nb, x} w_{N1b}^{nb kb} w_{P2}^{x kx} w_{P1}^{nb ka}
//               sum_{na} w_{N1a}^{na ka} Z[na, nb, x],
// so the forward transform is
//   pass A  per column (nb, x): a length-N1a FFT over na (stride BLK), then the
//           factor w_{P1}^{nb ka};
//   pass B  per block (one ka): the N1b x P2 two-dimensional FFT of its BLK
//           contiguous points, the product with the kernel spectrum, the
//           inverse two-dimensional FFT and the factor w_{P1}^{-nb ka};
//   pass C  per column: the inverse length-N1a FFT.
// Forward FFTs leave their output in bit-reversed order and the inverses take
// it back, so no permutation pass is needed; the spectrum (FP64 on the host,
// scaled by 1/P) is stored in the same order. The depth axis is reversed on
// scatter as in the shared-memory evaluator, so the correlation is a
// convolution and G_q[s] is read at (q, s).
//
// Only rows that can hold a bin are loaded by pass A (row 0 and rows >= P1 -
// maxr after the reversal) and only rows q <= maxr are stored by pass C.
#pragma once

#include "kernels.cuh"

namespace tfi {
namespace dev {

struct BigItem {
    int64_t off;       // offset of the item's P-point array in the batch buffer (complex elements)
    int64_t spec_off;  // offset of its size class's spectrum (complex elements)
    int32_t kb, ke;    // the table's bins
    int32_t pair;      // channel pair: channels 2 pair and 2 pair + 1
    int32_t maxr;      // largest depth among the bins (grid units)
};

// Geometry of one size class: log2 of P1 (outer), P2 (inner), N1a (column length)
// and N1b (block rows).
struct BigGeom {
    int lp1, lp2, lnA, lp1b;
};

constexpr int kBigTwLog = 26;  // largest P1 the twiddle tables cover

// exp(-2 pi i m / P1) for 0 <= m < P1 = 2^lp1 <= 2^26, from two FP32 tables filled in
// FP64 on the host: hi[j] = exp(-2 pi i j / 2^13), lo[j] = exp(-2 pi i j / 2^26)
__device__ __forceinline__ float2 big_twiddle(int64_t m, int lp1, const float2 *__restrict__ hi,
                                              const float2 *__restrict__ lo) {
    const int64_t M = m << (kBigTwLog - lp1);
    return cmul(__ldg(hi + (M >> 13)), __ldg(lo + (M & 8191)));
}

__device__ __forceinline__ int brev_bits(int v, int bits) { return bits == 0 ? 0 : int(__brev(unsigned(v)) >> (32 - bits)); }

// Zero the rows of every item's array that pass A reads (row block na = 0 and the
// blocks na >= na_lo that can hold a reversed depth); one grid row per item.
__global__ void big_zero(const BigItem *__restrict__ items, BigGeom g, float2 *__restrict__ buf) {
    const BigItem it = items[blockIdx.y];
    const int64_t BLK = int64_t(1) << (g.lp1b + g.lp2), P1 = int64_t(1) << g.lp1;
    const int64_t na_lo = (P1 - it.maxr) >> g.lp1b;
    const int64_t NA = int64_t(1) << g.lnA;
    float4 *a = reinterpret_cast<float4 *>(buf + it.off);
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    // two float2 per float4: block 0 and blocks [na_lo, NA)
    const int64_t h = BLK / 2;
    const int64_t n0 = h, n1 = (NA - na_lo) * h;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n0 + n1; i += int64_t(gridDim.x) * blockDim.x)
        a[i < n0 ? i : na_lo * h + (i - n0)] = z;
}

// Bin sums into the reversed-depth positions: channels 2 pair, 2 pair + 1 as one complex value.
__global__ void big_scatter(const BigItem *__restrict__ items, BigGeom g, const int32_t *__restrict__ key_r,
                            const int32_t *__restrict__ key_x, int d, const float *__restrict__ kbuf,
                            float2 *__restrict__ buf) {
    const BigItem it = items[blockIdx.y];
    const int64_t P1 = int64_t(1) << g.lp1;
    const int ch = 2 * it.pair;
    for (int k = it.kb + blockIdx.x * blockDim.x + threadIdx.x; k < it.ke; k += gridDim.x * blockDim.x) {
        const float re = kbuf[int64_t(k) * d + ch];
        const float im = ch + 1 < d ? kbuf[int64_t(k) * d + ch + 1] : 0.f;
        const int64_t pos = ((P1 - key_r[k]) & (P1 - 1)) * (int64_t(1) << g.lp2) + key_x[k];
        buf[it.off + pos] = make_float2(re, im);
    }
}

// Table values at the bins (depth q, coordinate s) after pass C.
__global__ void big_gather(const BigItem *__restrict__ items, BigGeom g, const int32_t *__restrict__ key_r,
                           const int32_t *__restrict__ key_x, int d, const float2 *__restrict__ buf,
                           float *__restrict__ vbuf) {
    const BigItem it = items[blockIdx.y];
    const int ch = 2 * it.pair;
    for (int k = it.kb + blockIdx.x * blockDim.x + threadIdx.x; k < it.ke; k += gridDim.x * blockDim.x) {
        const float2 v = buf[it.off + (int64_t(key_r[k]) << g.lp2) + key_x[k]];
        vbuf[int64_t(k) * d + ch] = v.x;
        if (ch + 1 < d) vbuf[int64_t(k) * d + ch + 1] = v.y;
    }
}

// Pass A (INV = false) and pass C (INV = true): 2^lcg adjacent columns per CTA, the
// length-N1a FFT over na in shared memory (element (na, c) at na 2^lcg + c). Columns
// per CTA are chosen so that a CTA holds about 2^13 points.
template <bool INV>
__global__ void __launch_bounds__(256) big_columns(const BigItem *__restrict__ items, BigGeom g, int lcg,
                                                   float2 *__restrict__ buf, const float2 *__restrict__ tw,
                                                   const float2 *__restrict__ tw_hi, const float2 *__restrict__ tw_lo) {
    extern __shared__ float2 Z[];
    const int CG = 1 << lcg;
    const int NA = 1 << g.lnA;
    const int64_t BLK = int64_t(1) << (g.lp1b + g.lp2);
    const int64_t per = BLK >> lcg;
    const BigItem it = items[blockIdx.x / per];
    const int64_t col0 = (blockIdx.x % per) << lcg;
    float2 *a = buf + it.off;
    const int64_t P1 = int64_t(1) << g.lp1;
    const int padnp = padded_size(NA << lcg);
    if (!INV) {
        // rows that can hold a bin: na = 0 and na >= na_lo; the rest are zero
        const int na_lo = int((P1 - it.maxr) >> g.lp1b);
        for (int e = threadIdx.x; e < (NA << lcg); e += blockDim.x) {
            const int na = e >> lcg, c = e & (CG - 1);
            Z[padded(e)] = (na == 0 || na >= na_lo) ? a[int64_t(na) * BLK + col0 + c] : make_float2(0.f, 0.f);
        }
    } else {
        for (int e = threadIdx.x; e < (NA << lcg); e += blockDim.x) {
            const int na = e >> lcg, c = e & (CG - 1);
            Z[padded(e)] = a[int64_t(na) * BLK + col0 + c];
        }
    }
    __syncthreads();
    if (!INV) {
        fft_axis<false>(Z, padnp, 1, g.lnA, CG, lcg, 1, true, tw, false);
        // slot s holds frequency ka = brev(s); column (nb, x) takes w_{P1}^{nb ka}
        for (int e = threadIdx.x; e < (NA << lcg); e += blockDim.x) {
            const int s = e >> lcg, c = e & (CG - 1);
            const int64_t nb = (col0 + c) >> g.lp2;
            const int64_t m = (nb * brev_bits(s, g.lnA)) & (P1 - 1);
            a[int64_t(s) * BLK + col0 + c] = m ? cmul(Z[padded(e)], big_twiddle(m, g.lp1, tw_hi, tw_lo)) : Z[padded(e)];
        }
    } else {
        fft_axis<true>(Z, padnp, 1, g.lnA, CG, lcg, 1, true, tw, false);
        // only depths q <= maxr are read back
        const int na_hi = it.maxr >> g.lp1b;
        for (int e = threadIdx.x; e < (NA << lcg); e += blockDim.x) {
            const int na = e >> lcg, c = e & (CG - 1);
            if (na <= na_hi) a[int64_t(na) * BLK + col0 + c] = Z[padded(e)];
        }
    }
}

// Pass B: 2^lnb consecutive blocks (consecutive ka slots) per CTA, each in its own
// padded shared-memory array: the N1b x P2 forward FFT, the product with that block's
// spectrum, the inverse FFT and the factor w_{P1}^{-nb ka}.
// CTAs run block-major (every item's blocks s0 .. s0 + 2^lnb - 1 next to each other): the
// items of a launch share their size class's spectrum, whose blocks then come from L2.
__global__ void __launch_bounds__(256) big_blocks(const BigItem *__restrict__ items, int n_items, BigGeom g, int lnb,
                                                  float2 *__restrict__ buf, const float2 *__restrict__ spectra,
                                                  const float2 *__restrict__ tw, const float2 *__restrict__ tw_hi,
                                                  const float2 *__restrict__ tw_lo) {
    extern __shared__ float2 Z[];
    const int lb = g.lp1b + g.lp2;
    const int BLK = 1 << lb, P2 = 1 << g.lp2, NBK = 1 << lnb;
    const BigItem it = items[blockIdx.x % n_items];
    const int s0 = int(blockIdx.x / n_items) << lnb;
    float2 *a = buf + it.off + int64_t(s0) * BLK;
    const int padnp = padded_size(BLK);
    for (int e = threadIdx.x; e < (BLK << lnb); e += blockDim.x) Z[(e >> lb) * padnp + padded(e & (BLK - 1))] = a[e];
    __syncthreads();
    const float2 *S = spectra + it.spec_off + int64_t(s0) * BLK;
    if (g.lp1b > 0) {
        fft_axis<false>(Z, padnp, NBK, g.lp2, 1, g.lp1b, P2, false, tw, false);
        fft_axis<false>(Z, padnp, NBK, g.lp1b, P2, g.lp2, 1, true, tw, true);
        fused_bottom(Z, padnp, NBK, g.lp1b, P2, g.lp2, 1, true, S, BLK);
        fft_axis<true>(Z, padnp, NBK, g.lp1b, P2, g.lp2, 1, true, tw, true);
        fft_axis<true>(Z, padnp, NBK, g.lp2, 1, g.lp1b, P2, false, tw, false);
    } else {
        fft_axis<false>(Z, padnp, NBK, g.lp2, 1, 0, P2, false, tw, true);
        fused_bottom(Z, padnp, NBK, g.lp2, 1, 0, P2, false, S, BLK);
        fft_axis<true>(Z, padnp, NBK, g.lp2, 1, 0, P2, false, tw, true);
    }
    const int64_t P1 = int64_t(1) << g.lp1;
    for (int e = threadIdx.x; e < (BLK << lnb); e += blockDim.x) {
        const int q = e >> lb, el = e & (BLK - 1);
        const int64_t ka = brev_bits(s0 + q, g.lnA);
        const int64_t m = ((int64_t(el >> g.lp2)) * ka) & (P1 - 1);
        const float2 v = Z[q * padnp + padded(el)];
        a[e] = m ? cmulc(v, big_twiddle(m, g.lp1, tw_hi, tw_lo)) : v;
    }
}

// Columns per CTA (log2) for passes A and C, and blocks per CTA (log2) for pass B: about
// 2^13 points per CTA.
__host__ __device__ inline int big_lcg(BigGeom g) {
    int l = 13 - g.lnA;
    if (l < 1) l = 1;
    if (l > g.lp1b + g.lp2) l = g.lp1b + g.lp2;
    return l;
}
__host__ __device__ inline int big_lnb(BigGeom g) {
    int l = 13 - (g.lp1b + g.lp2);
    if (l < 0) l = 0;
    if (l > g.lnA) l = g.lnA;
    return l;
}

}  // namespace dev
}  // namespace tfi
