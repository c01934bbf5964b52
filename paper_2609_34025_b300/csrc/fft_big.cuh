// Cross tables and corrections too large for one CTA's shared memory (P = P1 P2
// grid points with P > 2^14): the circular correlation of Eq.
// "stad-2d-convolution" (Eq. "stad-E" for a correction) evaluated by a four-step
// FFT through a global-memory buffer, one P-point array per (table, plane of four
// channels): each point is one 16-byte element holding two channel pairs as
// (re0, re1, im0, im1), transformed on the paired FP32 instructions of the
// shared-memory FFT (fft_x2.cuh), in its XOR-swizzled shared-memory layout.
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

#include "fft_x2.cuh"

namespace tfi {
namespace dev {

struct BigItem {
    int64_t off;       // offset of the item's P-point array in the batch buffer (16-byte elements)
    int64_t spec_off;  // offset of its size class's spectrum (complex elements)
    int32_t kb, ke;    // the table's bins
    int32_t plane;     // channels 4 plane .. 4 plane + 3 (pairs (4p, 4p+1) and (4p+2, 4p+3))
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
__global__ void big_zero(const BigItem *__restrict__ items, BigGeom g, ulonglong2 *__restrict__ buf) {
    const BigItem it = items[blockIdx.y];
    const int64_t BLK = int64_t(1) << (g.lp1b + g.lp2), P1 = int64_t(1) << g.lp1;
    const int64_t na_lo = (P1 - it.maxr) >> g.lp1b;
    const int64_t NA = int64_t(1) << g.lnA;
    ulonglong2 *a = buf + it.off;
    const ulonglong2 z = make_ulonglong2(0ull, 0ull);
    const int64_t n0 = BLK, n1 = (NA - na_lo) * BLK;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n0 + n1; i += int64_t(gridDim.x) * blockDim.x)
        a[i < n0 ? i : na_lo * BLK + (i - n0)] = z;
}

// Bin sums into the reversed-depth positions: the plane's four channels as one element.
__global__ void big_scatter(const BigItem *__restrict__ items, BigGeom g, const int32_t *__restrict__ key_r,
                            const int32_t *__restrict__ key_x, int d, const float *__restrict__ kbuf,
                            ulonglong2 *__restrict__ buf) {
    const BigItem it = items[blockIdx.y];
    const int64_t P1 = int64_t(1) << g.lp1;
    const int c = 4 * it.plane;
    const bool vec = (d & 3) == 0;
    for (int k = it.kb + blockIdx.x * blockDim.x + threadIdx.x; k < it.ke; k += gridDim.x * blockDim.x) {
        float4 q;
        if (vec) {
            q = __ldg(reinterpret_cast<const float4 *>(kbuf + int64_t(k) * d + c));
        } else {
            const float *row = kbuf + int64_t(k) * d;
            q.x = c < d ? row[c] : 0.f;
            q.y = c + 1 < d ? row[c + 1] : 0.f;
            q.z = c + 2 < d ? row[c + 2] : 0.f;
            q.w = c + 3 < d ? row[c + 3] : 0.f;
        }
        const int64_t pos = ((P1 - key_r[k]) & (P1 - 1)) * (int64_t(1) << g.lp2) + key_x[k];
        buf[it.off + pos] = make_ulonglong2(vpack(q.x, q.z), vpack(q.y, q.w));
    }
}

// Table values at the bins (depth q, coordinate s) after pass C.
__global__ void big_gather(const BigItem *__restrict__ items, BigGeom g, const int32_t *__restrict__ key_r,
                           const int32_t *__restrict__ key_x, int d, const ulonglong2 *__restrict__ buf,
                           float *__restrict__ vbuf) {
    const BigItem it = items[blockIdx.y];
    const int c = 4 * it.plane;
    const bool vec = (d & 3) == 0;
    for (int k = it.kb + blockIdx.x * blockDim.x + threadIdx.x; k < it.ke; k += gridDim.x * blockDim.x) {
        const ulonglong2 v = buf[it.off + (int64_t(key_r[k]) << g.lp2) + key_x[k]];
        float4 o;
        vunpack(v.x, o.x, o.z);
        vunpack(v.y, o.y, o.w);
        if (vec) {
            *reinterpret_cast<float4 *>(vbuf + int64_t(k) * d + c) = o;
        } else {
            float *row = vbuf + int64_t(k) * d;
            if (c < d) row[c] = o.x;
            if (c + 1 < d) row[c + 1] = o.y;
            if (c + 2 < d) row[c + 2] = o.z;
            if (c + 3 < d) row[c + 3] = o.w;
        }
    }
}

// Pass A (INV = false) and pass C (INV = true): 2^lcg adjacent columns per CTA, the
// length-N1a FFT over na in shared memory (element (na, c) at slot swz(na 2^lcg + c)).
template <bool INV>
__global__ void __launch_bounds__(256) big_columns(const BigItem *__restrict__ items, BigGeom g, int lcg,
                                                   ulonglong2 *__restrict__ buf, const float2 *__restrict__ tw,
                                                   const float2 *__restrict__ tw_hi, const float2 *__restrict__ tw_lo) {
    extern __shared__ ulonglong2 Zc[];
    const int CG = 1 << lcg;
    const int NA = 1 << g.lnA;
    const int NP = NA << lcg;
    const int64_t BLK = int64_t(1) << (g.lp1b + g.lp2);
    const int64_t per = BLK >> lcg;
    const BigItem it = items[blockIdx.x / per];
    const int64_t col0 = (blockIdx.x % per) << lcg;
    ulonglong2 *a = buf + it.off;
    const int64_t P1 = int64_t(1) << g.lp1;
    if (!INV) {
        // rows that can hold a bin: na = 0 and na >= na_lo; the rest are zero
        const int na_lo = int((P1 - it.maxr) >> g.lp1b);
        for (int e = threadIdx.x; e < NP; e += blockDim.x) {
            const int na = e >> lcg, c = e & (CG - 1);
            Zc[swz(e)] = (na == 0 || na >= na_lo) ? a[int64_t(na) * BLK + col0 + c] : make_ulonglong2(0ull, 0ull);
        }
    } else {
        for (int e = threadIdx.x; e < NP; e += blockDim.x) {
            const int na = e >> lcg, c = e & (CG - 1);
            Zc[swz(e)] = a[int64_t(na) * BLK + col0 + c];
        }
    }
    __syncthreads();
    if (!INV) {
        fft_axis_x2<false>(Zc, NP, 1, g.lnA, CG, lcg, 1, true, tw, false);
        // slot s holds frequency ka = brev(s); column (nb, x) takes w_{P1}^{nb ka}
        for (int e = threadIdx.x; e < NP; e += blockDim.x) {
            const int s = e >> lcg, c = e & (CG - 1);
            const int64_t nb = (col0 + c) >> g.lp2;
            const int64_t m = (nb * brev_bits(s, g.lnA)) & (P1 - 1);
            const ulonglong2 q = Zc[swz(e)];
            Cx2 v{q.x, q.y};
            if (m) v = cx_mul(v, cx_bcast(big_twiddle(m, g.lp1, tw_hi, tw_lo)));
            a[int64_t(s) * BLK + col0 + c] = make_ulonglong2(v.re, v.im);
        }
    } else {
        fft_axis_x2<true>(Zc, NP, 1, g.lnA, CG, lcg, 1, true, tw, false);
        // only depths q <= maxr are read back
        const int na_hi = it.maxr >> g.lp1b;
        for (int e = threadIdx.x; e < NP; e += blockDim.x) {
            const int na = e >> lcg, c = e & (CG - 1);
            if (na <= na_hi) a[int64_t(na) * BLK + col0 + c] = Zc[swz(e)];
        }
    }
}

// Pass B: 2^lnb consecutive blocks (consecutive ka slots) per CTA, one plane each: the
// N1b x P2 forward FFT, the product with that block's spectrum, the inverse FFT and the
// factor w_{P1}^{-nb ka}. CTAs run block-major (every item's blocks s0 .. next to each
// other): the items of a launch share their size class's spectrum, whose blocks then
// come from L2.
__global__ void __launch_bounds__(256) big_blocks(const BigItem *__restrict__ items, int n_items, BigGeom g, int lnb,
                                                  ulonglong2 *__restrict__ buf, const float2 *__restrict__ spectra,
                                                  const float2 *__restrict__ tw, const ulonglong2 *__restrict__ twb,
                                                  const float2 *__restrict__ tw_hi, const float2 *__restrict__ tw_lo) {
    extern __shared__ ulonglong2 Zb[];
    const int lb = g.lp1b + g.lp2;
    const int BLK = 1 << lb, P2 = 1 << g.lp2, NBK = 1 << lnb;
    const BigItem it = items[blockIdx.x % n_items];
    const int s0 = int(blockIdx.x / n_items) << lnb;
    ulonglong2 *a = buf + it.off + int64_t(s0) * BLK;
    for (int e = threadIdx.x; e < (BLK << lnb); e += blockDim.x) Zb[(e >> lb) * BLK + swz(e & (BLK - 1))] = a[e];
    __syncthreads();
    const float2 *S = spectra + it.spec_off + int64_t(s0) * BLK;
    if (g.lp2 == 0) {
        // one axis of 2^lp1b points per block
        fft_1d_x2(Zb, BLK, NBK, g.lp1b, tw, twb, S, BLK);
    } else if (g.lp1b > 0) {
        fft_axis_x2<false>(Zb, BLK, NBK, g.lp2, 1, g.lp1b, P2, false, tw, false);
        fft_axis_x2<false>(Zb, BLK, NBK, g.lp1b, P2, g.lp2, 1, true, tw, true);
        fused_bottom_x2(Zb, BLK, NBK, g.lp1b, P2, g.lp2, 1, true, S, BLK);
        fft_axis_x2<true>(Zb, BLK, NBK, g.lp1b, P2, g.lp2, 1, true, tw, true);
        fft_axis_x2<true>(Zb, BLK, NBK, g.lp2, 1, g.lp1b, P2, false, tw, false);
    } else {
        fft_1d_x2(Zb, BLK, NBK, g.lp2, tw, twb, S, BLK);
    }
    const int64_t P1 = int64_t(1) << g.lp1;
    for (int e = threadIdx.x; e < (BLK << lnb); e += blockDim.x) {
        const int q = e >> lb, el = e & (BLK - 1);
        const int64_t ka = brev_bits(s0 + q, g.lnA);
        const int64_t m = ((int64_t(el >> g.lp2)) * ka) & (P1 - 1);
        const ulonglong2 z = Zb[q * BLK + swz(el)];
        Cx2 v{z.x, z.y};
        if (m) v = cx_mulc(v, cx_bcast(big_twiddle(m, g.lp1, tw_hi, tw_lo)));
        a[e] = make_ulonglong2(v.re, v.im);
    }
}

// Columns per CTA (log2) for passes A and C, and blocks per CTA (log2) for pass B: 2^12
// points (64 KB) per CTA, 2^13 where a column or a block alone needs it.
__host__ __device__ inline int big_lcg(BigGeom g) {
    int l = 12 - g.lnA;
    if (l < 1) l = 1;
    if (l > g.lp1b + g.lp2) l = g.lp1b + g.lp2;
    return l;
}
__host__ __device__ inline int big_lnb(BigGeom g) {
    int l = 12 - (g.lp1b + g.lp2);
    if (l < 0) l = 0;
    if (l > g.lnA) l = g.lnA;
    return l;
}

}  // namespace dev
}  // namespace tfi
