// FFT job kernel for two channel pairs per element (the same job as fft_kernel:
// the cross table G = K * A of Eq. "stad-2d-convolution", or a correction
// E_alpha of Eq. "stad-E", as a circular correlation in shared memory).
//
// Each shared-memory element is 16 bytes and holds one complex point of two
// channel pairs, stored as (re0, re1, im0, im1): pair 0 carries channels
// (c, c+1) as re + i im, pair 1 channels (c+2, c+3). Both pairs see the same
// butterflies and twiddles, so
//   - every shared-memory access moves both pairs (one 16-byte load or store),
//   - additions and multiplications run on the paired FP32 instructions of
//     sm_100+ (add / sub / mul / fma .rn.f32x2), one instruction for both pairs,
//   - each twiddle is generated once for the two pairs.
// The butterfly schedule is fft_kernel's: radix-8 decimation in frequency
// (natural -> bit-reversed) ahead of the spectrum product, decimation in time
// back, the span-1 pass fused with the product.
//
// Layout: element e of a plane sits at slot e ^ ((e >> 3) & 7) (no padding).
// A 16-byte access is served eight lanes per shared-memory wavefront; with this
// swizzle the eight lanes of every quarter warp fall on distinct 16-byte bank
// groups in all passes of a one-dimensional table: lanes that differ in bits
// 0..2 of e keep them distinct, lanes that differ only in bits 3..5 (the span-1
// pass) have them folded into bits 0..2.
#pragma once

#include "kernels.cuh"

namespace tfi {
namespace dev {

typedef unsigned long long f32x2;  // two FP32 lanes in one 64-bit register pair

__device__ __forceinline__ f32x2 vpack(float a, float b) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void vunpack(f32x2 v, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f32x2 vadd(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 vsub(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 vmul(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 vfma(f32x2 a, f32x2 b, f32x2 c) {  // a * b + c
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// one complex point of two channel pairs
struct Cx2 {
    f32x2 re, im;
};

__device__ __forceinline__ Cx2 cx_add(Cx2 a, Cx2 b) { return Cx2{vadd(a.re, b.re), vadd(a.im, b.im)}; }
__device__ __forceinline__ Cx2 cx_sub(Cx2 a, Cx2 b) { return Cx2{vsub(a.re, b.re), vsub(a.im, b.im)}; }
// a * w, w broadcast to both lanes
__device__ __forceinline__ Cx2 cx_mul(Cx2 a, Cx2 w) {
    return Cx2{vsub(vmul(a.re, w.re), vmul(a.im, w.im)), vfma(a.re, w.im, vmul(a.im, w.re))};
}
// a * conj(w)
__device__ __forceinline__ Cx2 cx_mulc(Cx2 a, Cx2 w) {
    return Cx2{vfma(a.im, w.im, vmul(a.re, w.re)), vsub(vmul(a.im, w.re), vmul(a.re, w.im))};
}
__device__ __forceinline__ Cx2 cx_bcast(float2 w) {
    f32x2 r, i;
    asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(w.x));
    asm("mov.b64 %0, {%1, %1};" : "=l"(i) : "f"(w.y));
    return Cx2{r, i};
}

constexpr f32x2 kSqrtHalf2 = 0x3F3504F33F3504F3ull;   // (1/sqrt2, 1/sqrt2)
constexpr f32x2 kNSqrtHalf2 = 0xBF3504F3BF3504F3ull;  // (-1/sqrt2, -1/sqrt2)

__device__ __forceinline__ int swz(int e) { return e ^ ((e >> 3) & 7); }

// Decimation-in-frequency butterfly (a, b) -> (a + b, (a - b) w) with the
// constant twiddle w = exp(-2 pi i j / (2 dt)), dt <= 4 (dt, j constant after
// unrolling).
__device__ __forceinline__ void bfly_dif(Cx2 &a, Cx2 &b, int dt, int j) {
    const Cx2 s = cx_add(a, b);
    if (j == 0) {
        b = cx_sub(a, b);
    } else if (dt == 2 || (dt == 4 && j == 2)) {  // w = -i: (d.im, -d.re)
        b = Cx2{vsub(a.im, b.im), vsub(b.re, a.re)};
    } else {
        const Cx2 d = cx_sub(a, b);
        const f32x2 p = vadd(d.re, d.im), m = vsub(d.im, d.re);
        if (j == 1)  // w = (1 - i)/sqrt2: (p, m)/sqrt2
            b = Cx2{vmul(p, kSqrtHalf2), vmul(m, kSqrtHalf2)};
        else  // j == 3, w = (-1 - i)/sqrt2: (m, -p)/sqrt2
            b = Cx2{vmul(m, kSqrtHalf2), vmul(p, kNSqrtHalf2)};
    }
    a = s;
}

// Decimation-in-time butterfly (a, b) -> (a + x, a - x), x = b conj(w), the
// inverse of bfly_dif up to the factor 2.
__device__ __forceinline__ void bfly_dit(Cx2 &a, Cx2 &b, int dt, int j) {
    if (j == 0) {
        const Cx2 s = cx_add(a, b);
        b = cx_sub(a, b);
        a = s;
    } else if (dt == 2 || (dt == 4 && j == 2)) {  // conj(w) = +i: x = (-b.im, b.re)
        const Cx2 s = Cx2{vsub(a.re, b.im), vadd(a.im, b.re)};
        b = Cx2{vadd(a.re, b.im), vsub(a.im, b.re)};
        a = s;
    } else if (j == 1) {  // conj(w) = (1 + i)/sqrt2: x = (q, r)/sqrt2, q = re - im, r = re + im
        const f32x2 q = vsub(b.re, b.im), r = vadd(b.re, b.im);
        const Cx2 s = Cx2{vfma(q, kSqrtHalf2, a.re), vfma(r, kSqrtHalf2, a.im)};
        b = Cx2{vfma(q, kNSqrtHalf2, a.re), vfma(r, kNSqrtHalf2, a.im)};
        a = s;
    } else {  // j == 3, conj(w) = (-1 + i)/sqrt2: x = (-q, r)/sqrt2, q = re + im, r = re - im
        const f32x2 q = vadd(b.re, b.im), r = vsub(b.re, b.im);
        const Cx2 s = Cx2{vfma(q, kNSqrtHalf2, a.re), vfma(r, kSqrtHalf2, a.im)};
        b = Cx2{vfma(q, kSqrtHalf2, a.re), vfma(r, kNSqrtHalf2, a.im)};
        a = s;
    }
}

// 2^RL-point DFT in registers, natural order in, bit-reversed order out.
template <int RL>
__device__ __forceinline__ void dft_dif_x2(Cx2 *v) {
    constexpr int R = 1 << RL;
#pragma unroll
    for (int st = RL - 1; st >= 0; --st) {
        const int dt = 1 << st;
#pragma unroll
        for (int t = 0; t < R; ++t)
            if (!(t & dt)) bfly_dif(v[t], v[t + dt], dt, t & (dt - 1));
    }
}

// Inverse of dft_dif_x2 up to the factor 2^RL.
template <int RL>
__device__ __forceinline__ void idft_dit_x2(Cx2 *v) {
    constexpr int R = 1 << RL;
#pragma unroll
    for (int st = 0; st < RL; ++st) {
        const int dt = 1 << st;
#pragma unroll
        for (int t = 0; t < R; ++t)
            if (!(t & dt)) bfly_dit(v[t], v[t + dt], dt, t & (dt - 1));
    }
}

// Multiplies the bit-reversed DFT outputs by w^k (slot brev(k)), w = w8^(8/R),
// generating each power next to its use (CONJ: by the conjugates).
template <bool CONJ>
__device__ __forceinline__ Cx2 tw_mul(Cx2 a, Cx2 w) { return CONJ ? cx_mulc(a, w) : cx_mul(a, w); }

template <int RL, bool CONJ>
__device__ __forceinline__ void apply_twiddles(Cx2 *v, Cx2 w8) {
    if (RL == 3) {
        const Cx2 w2 = cx_mul(w8, w8), w3 = cx_mul(w8, w2), w4 = cx_mul(w2, w2);
        v[4] = tw_mul<CONJ>(v[4], w8);
        v[2] = tw_mul<CONJ>(v[2], w2);
        v[6] = tw_mul<CONJ>(v[6], w3);
        v[1] = tw_mul<CONJ>(v[1], w4);
        v[5] = tw_mul<CONJ>(v[5], cx_mul(w8, w4));
        v[3] = tw_mul<CONJ>(v[3], cx_mul(w2, w4));
        v[7] = tw_mul<CONJ>(v[7], cx_mul(w3, w4));
    } else if (RL == 2) {
        const Cx2 w = cx_mul(w8, w8), w2 = cx_mul(w, w);
        v[2] = tw_mul<CONJ>(v[2], w);
        v[1] = tw_mul<CONJ>(v[1], w2);
        v[3] = tw_mul<CONJ>(v[3], cx_mul(w, w2));
    } else {
        const Cx2 w4 = cx_mul(w8, w8);
        v[1] = tw_mul<CONJ>(v[1], cx_mul(w4, w4));
    }
}

// Slots of the R elements e0 + t H of one group.
template <int R>
__device__ __forceinline__ void group_slots(int e0, int H, int *adr) {
    if ((H & 63) == 0) {  // bits 0..5 of e are those of e0 for every t
        const int a0 = swz(e0);
#pragma unroll
        for (int t = 0; t < R; ++t) adr[t] = a0 + t * H;
    } else {
#pragma unroll
        for (int t = 0; t < R; ++t) adr[t] = swz(e0 + t * H);
    }
}

// One radix-2^RL pass (same group structure and twiddles as fft_pass) over
// nplane planes of NP elements.
template <bool INV, int RL>
__device__ __forceinline__ void fft_pass_x2(ulonglong2 *Z, int NP, int nplane, int ln, int lh_lo, int es, int llog,
                                            int ls, bool line_fast, const float2 *__restrict__ tw) {
    constexpr int R = 1 << RL;
    const int glog = ln - RL;
    const int total = nplane << (llog + glog);
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
        ulonglong2 *Zp = Z + p * NP;
        const int e0 = line * ls + base * es, H = es << lh_lo;
        int adr[R];
        group_slots<R>(e0, H, adr);
        Cx2 v[R];
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const ulonglong2 q = Zp[adr[t]];
            v[t] = Cx2{q.x, q.y};
        }
        // w^k, w = exp(-2 pi i o / (R h)), from the per-level entry exp(-2 pi i o / (8 h))
        Cx2 w8;
        if (lh_lo > 0) w8 = cx_bcast(__ldg(tw + (1 << lh_lo) + o));
        if (!INV) {
            dft_dif_x2<RL>(v);
            if (lh_lo > 0) apply_twiddles<RL, false>(v, w8);
        } else {
            if (lh_lo > 0) apply_twiddles<RL, true>(v, w8);
            idft_dit_x2<RL>(v);
        }
#pragma unroll
        for (int t = 0; t < R; ++t) Zp[adr[t]] = make_ulonglong2(v[t].re, v[t].im);
    }
    __syncthreads();
}

template <bool INV>
__device__ __forceinline__ void fft_axis_x2(ulonglong2 *Z, int NP, int nplane, int ln, int es, int llog, int ls,
                                            bool line_fast, const float2 *__restrict__ tw, bool skip_bottom) {
    if (ln == 0) return;
    const int full = ln / 3, rem = ln - 3 * full;
    const bool do_rem = rem && !(skip_bottom && full == 0);
    if (!INV) {
        if (do_rem) {
            if (rem == 2) fft_pass_x2<false, 2>(Z, NP, nplane, ln, ln - 2, es, llog, ls, line_fast, tw);
            else fft_pass_x2<false, 1>(Z, NP, nplane, ln, ln - 1, es, llog, ls, line_fast, tw);
        }
        for (int k = 0; k < full; ++k) {
            const int lh = ln - rem - 3 * (k + 1);
            if (skip_bottom && lh == 0) break;
            fft_pass_x2<false, 3>(Z, NP, nplane, ln, lh, es, llog, ls, line_fast, tw);
        }
    } else {
        for (int k = full - 1; k >= 0; --k) {
            const int lh = ln - rem - 3 * (k + 1);
            if (skip_bottom && lh == 0) continue;
            fft_pass_x2<true, 3>(Z, NP, nplane, ln, lh, es, llog, ls, line_fast, tw);
        }
        if (do_rem) {
            if (rem == 2) fft_pass_x2<true, 2>(Z, NP, nplane, ln, ln - 2, es, llog, ls, line_fast, tw);
            else fft_pass_x2<true, 1>(Z, NP, nplane, ln, ln - 1, es, llog, ls, line_fast, tw);
        }
    }
}

// Span-1 pass of the innermost axis, forward and inverse, with the product by
// the kernel spectrum (one spectrum value per point, shared by both pairs).
// s_plane: offset between the spectra of consecutive planes (0: one spectrum for all)
template <int RL>
__device__ __forceinline__ void fused_bottom_pass_x2(ulonglong2 *Z, int NP, int nplane, int ln, int es, int llog,
                                                     int ls, bool line_fast, const float2 *__restrict__ S,
                                                     int s_plane) {
    constexpr int R = 1 << RL;
    const int glog = ln - RL;
    const int total = nplane << (llog + glog);
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
        ulonglong2 *Zp = Z + p * NP;
        const int e0 = line * ls + (g << RL) * es;
        int adr[R];
        group_slots<R>(e0, es, adr);
        Cx2 v[R];
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const ulonglong2 q = Zp[adr[t]];
            v[t] = Cx2{q.x, q.y};
        }
        dft_dif_x2<RL>(v);
        const float2 *Sp = S + p * s_plane;
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = cx_mul(v[q], cx_bcast(__ldg(Sp + e0 + q * es)));
        idft_dit_x2<RL>(v);
#pragma unroll
        for (int t = 0; t < R; ++t) Zp[adr[t]] = make_ulonglong2(v[t].re, v[t].im);
    }
    __syncthreads();
}

__device__ __forceinline__ void fused_bottom_x2(ulonglong2 *Z, int NP, int nplane, int ln, int es, int llog, int ls,
                                                bool line_fast, const float2 *__restrict__ S, int s_plane = 0) {
    const int full = ln / 3, rem = ln - 3 * full;
    const int rl = full > 0 ? 3 : rem;
    if (rl == 3) fused_bottom_pass_x2<3>(Z, NP, nplane, ln, es, llog, ls, line_fast, S, s_plane);
    else if (rl == 2) fused_bottom_pass_x2<2>(Z, NP, nplane, ln, es, llog, ls, line_fast, S, s_plane);
    else fused_bottom_pass_x2<1>(Z, NP, nplane, ln, es, llog, ls, line_fast, S, s_plane);
}

// ---------------------------------------------------------------------------
// One-dimensional tables (a single axis of 2^ln points, element stride 1): the
// same passes with the span H = 2^LH a compile-time constant, so that a group's
// slots are one base plus constant offsets, and with the twiddles read from a
// table already broadcast to both lanes ((re, re, im, im) per entry). The
// spectrum stays at 8 bytes a point: a class's spectrum is read by all its CTAs
// and stays in L1 at that size (a broadcast copy, twice as large, did not).
// Slots for e = e0 + t H, e0 = (g >> LH) << (LH + RL) | o, o < H:
//   H >= 64: bits 0..5 of e are those of e0: swz(e0) + t H;
//   H == 8, radix 8: bits 3..5 of e are t: (e0 + 8 t) ^ t = (e0 ^ t) + 8 t;
//   H == 1, radix 8: e0 = 8 g, bits 3..5 are g & 7: e0 ^ (g & 7) ^ t;
//   otherwise swz(e0 + t H).
// ---------------------------------------------------------------------------
template <int RL, int LH>
__device__ __forceinline__ void slots_1d(int e0, int *adr) {
    constexpr int R = 1 << RL;
    if (LH >= 6) {
        const int a0 = swz(e0);
#pragma unroll
        for (int t = 0; t < R; ++t) adr[t] = a0 + t * (1 << LH);
    } else if (LH == 3 && RL == 3) {
#pragma unroll
        for (int t = 0; t < R; ++t) adr[t] = (e0 ^ t) + 8 * t;
    } else if (LH == 0 && RL == 3) {
        const int b = e0 ^ ((e0 >> 3) & 7);
#pragma unroll
        for (int t = 0; t < R; ++t) adr[t] = b ^ t;
    } else {
#pragma unroll
        for (int t = 0; t < R; ++t) adr[t] = swz(e0 + t * (1 << LH));
    }
}

__device__ __forceinline__ Cx2 ld_bcast(const ulonglong2 *__restrict__ p) {
    const ulonglong2 q = __ldg(p);
    return Cx2{q.x, q.y};
}

template <bool INV, int RL, int LH>
__device__ __forceinline__ void pass_1d_x2(ulonglong2 *Z, int NP, int nplane, int ln,
                                           const ulonglong2 *__restrict__ twb) {
    constexpr int R = 1 << RL, H = 1 << LH;
    const int glog = ln - RL;
    const int total = nplane << glog;
    const int gmask = (1 << glog) - 1;
    for (int w = threadIdx.x; w < total; w += blockDim.x) {
        const int g = w & gmask, p = w >> glog;
        const int o = g & (H - 1);
        const int e0 = ((g >> LH) << (LH + RL)) + o;
        ulonglong2 *Zp = Z + p * NP;
        int adr[R];
        slots_1d<RL, LH>(e0, adr);
        Cx2 v[R];
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const ulonglong2 q = Zp[adr[t]];
            v[t] = Cx2{q.x, q.y};
        }
        const Cx2 w8 = ld_bcast(twb + H + o);
        if (!INV) {
            dft_dif_x2<RL>(v);
            apply_twiddles<RL, false>(v, w8);
        } else {
            apply_twiddles<RL, true>(v, w8);
            idft_dit_x2<RL>(v);
        }
#pragma unroll
        for (int t = 0; t < R; ++t) Zp[adr[t]] = make_ulonglong2(v[t].re, v[t].im);
    }
    __syncthreads();
}

// a pass at span 2^lh (lh = 3, 6 or 9 for the tables of up to 2^12 points this
// kernel runs; any other span takes the general pass)
template <bool INV, int RL>
__device__ __forceinline__ void pass_1d_dispatch(ulonglong2 *Z, int NP, int nplane, int ln, int lh,
                                                 const float2 *__restrict__ tw, const ulonglong2 *__restrict__ twb) {
    if (lh == 3) pass_1d_x2<INV, RL, 3>(Z, NP, nplane, ln, twb);
    else if (lh == 6) pass_1d_x2<INV, RL, 6>(Z, NP, nplane, ln, twb);
    else if (lh == 9) pass_1d_x2<INV, RL, 9>(Z, NP, nplane, ln, twb);
    else fft_pass_x2<INV, RL>(Z, NP, nplane, ln, lh, 1, 0, 0, false, tw);
}

// span-1 pass with the spectrum product
template <int RL>
__device__ __forceinline__ void bottom_1d_x2(ulonglong2 *Z, int NP, int nplane, int ln,
                                             const float2 *__restrict__ S, int s_plane) {
    constexpr int R = 1 << RL;
    const int glog = ln - RL;
    const int total = nplane << glog;
    const int gmask = (1 << glog) - 1;
    for (int w = threadIdx.x; w < total; w += blockDim.x) {
        const int g = w & gmask, p = w >> glog;
        const int e0 = g << RL;
        ulonglong2 *Zp = Z + p * NP;
        int adr[R];
        slots_1d<RL, 0>(e0, adr);
        Cx2 v[R];
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const ulonglong2 q = Zp[adr[t]];
            v[t] = Cx2{q.x, q.y};
        }
        dft_dif_x2<RL>(v);
        const float2 *Sp = S + p * s_plane;
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = cx_mul(v[q], cx_bcast(__ldg(Sp + e0 + q)));
        idft_dit_x2<RL>(v);
#pragma unroll
        for (int t = 0; t < R; ++t) Zp[adr[t]] = make_ulonglong2(v[t].re, v[t].im);
    }
    __syncthreads();
}

// forward transform, spectrum product and inverse of a 2^ln-point table (ln >= 1); s_plane as in
// fused_bottom_pass_x2
__device__ __forceinline__ void fft_1d_x2(ulonglong2 *Z, int NP, int nplane, int ln, const float2 *__restrict__ tw,
                                          const ulonglong2 *__restrict__ twb, const float2 *__restrict__ S,
                                          int s_plane = 0) {
    const int full = ln / 3, rem = ln - 3 * full;
    if (full > 0) {
        if (rem == 2) pass_1d_dispatch<false, 2>(Z, NP, nplane, ln, ln - 2, tw, twb);
        else if (rem == 1) pass_1d_dispatch<false, 1>(Z, NP, nplane, ln, ln - 1, tw, twb);
        for (int k = 0; k < full - 1; ++k) pass_1d_dispatch<false, 3>(Z, NP, nplane, ln, ln - rem - 3 * (k + 1), tw, twb);
        bottom_1d_x2<3>(Z, NP, nplane, ln, S, s_plane);
        for (int k = full - 2; k >= 0; --k) pass_1d_dispatch<true, 3>(Z, NP, nplane, ln, ln - rem - 3 * (k + 1), tw, twb);
        if (rem == 2) pass_1d_dispatch<true, 2>(Z, NP, nplane, ln, ln - 2, tw, twb);
        else if (rem == 1) pass_1d_dispatch<true, 1>(Z, NP, nplane, ln, ln - 1, tw, twb);
    } else if (rem == 2) {
        bottom_1d_x2<2>(Z, NP, nplane, ln, S, s_plane);
    } else {
        bottom_1d_x2<1>(Z, NP, nplane, ln, S, s_plane);
    }
}

// One CTA per (job, up to 2 * nplane channel pairs starting at pair0): plane
// p holds pairs pair0 + 2p and pair0 + 2p + 1 (channels 2 pair0 + 4p .. + 3);
// channels at or beyond d ride as zeros.
__global__ void __launch_bounds__(256)
    fft_x2_kernel(const FftItem *__restrict__ items, const JobDev *__restrict__ jobs,
                  const int32_t *__restrict__ key_r, const int32_t *__restrict__ key_x, int d,
                  const float *__restrict__ kbuf, float *__restrict__ vbuf, const float2 *__restrict__ spectra,
                  const float2 *__restrict__ tw, const ulonglong2 *__restrict__ twb) {
    extern __shared__ ulonglong2 Zx[];
    const FftItem it = items[blockIdx.x];
    const JobDev jb = jobs[it.job];
    const int lp1 = jb.lp1, lp2 = jb.lp2;
    const int NP = 1 << (lp1 + lp2), P1 = 1 << lp1, P2 = 1 << lp2;
    const int nplane = (it.npair + 1) >> 1;
    for (int i = threadIdx.x; i < nplane * NP; i += blockDim.x) Zx[i] = make_ulonglong2(0ull, 0ull);
    __syncthreads();
    const int cbase = 2 * it.pair0;
    const int cend = min(d, 2 * (it.pair0 + it.npair));
    // whole planes move as one 16-byte access per key
    const bool vec_io = (d & 3) == 0 && (cbase & 3) == 0 && cend == cbase + 4 * nplane;
    const int nk = jb.ke - jb.kb;
    // scatter bin sums; depth reversed so the depth correlation becomes a convolution
    for (int t = threadIdx.x; t < nk * nplane; t += blockDim.x) {
        const int kk = t / nplane, p = t - kk * nplane;
        const int k = jb.kb + kk;
        const int c = cbase + 4 * p;
        float4 q;
        if (vec_io) {
            q = __ldg(reinterpret_cast<const float4 *>(kbuf + int64_t(k) * d + c));
        } else {
            const float *row = kbuf + int64_t(k) * d;
            q.x = c < cend ? row[c] : 0.f;
            q.y = c + 1 < cend ? row[c + 1] : 0.f;
            q.z = c + 2 < cend ? row[c + 2] : 0.f;
            q.w = c + 3 < cend ? row[c + 3] : 0.f;
        }
        const int pos = ((P1 - key_r[k]) & (P1 - 1)) * P2 + key_x[k];
        Zx[p * NP + swz(pos)] = make_ulonglong2(vpack(q.x, q.z), vpack(q.y, q.w));
    }
    __syncthreads();
    const float2 *S = spectra + jb.spec_off;
    if ((lp1 > 0) != (lp2 > 0)) {
        // one axis: 2^(lp1 + lp2) points at stride 1
        fft_1d_x2(Zx, NP, nplane, lp1 + lp2, tw, twb, S);
    } else if (lp1 > 0) {
        fft_axis_x2<false>(Zx, NP, nplane, lp2, 1, lp1, P2, false, tw, false);
        fft_axis_x2<false>(Zx, NP, nplane, lp1, P2, lp2, 1, true, tw, true);
        fused_bottom_x2(Zx, NP, nplane, lp1, P2, lp2, 1, true, S);
        fft_axis_x2<true>(Zx, NP, nplane, lp1, P2, lp2, 1, true, tw, true);
        fft_axis_x2<true>(Zx, NP, nplane, lp2, 1, lp1, P2, false, tw, false);
    } else {
        const Cx2 s0 = cx_bcast(__ldg(S));
        for (int p = threadIdx.x; p < nplane; p += blockDim.x) {
            const ulonglong2 q = Zx[p * NP];
            const Cx2 v = cx_mul(Cx2{q.x, q.y}, s0);
            Zx[p * NP] = make_ulonglong2(v.re, v.im);
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < nk * nplane; t += blockDim.x) {
        const int kk = t / nplane, p = t - kk * nplane;
        const int k = jb.kb + kk;
        const int c = cbase + 4 * p;
        const ulonglong2 q = Zx[p * NP + swz(key_r[k] * P2 + key_x[k])];
        float4 o;
        vunpack(q.x, o.x, o.z);
        vunpack(q.y, o.y, o.w);
        if (vec_io) {
            *reinterpret_cast<float4 *>(vbuf + int64_t(k) * d + c) = o;
        } else {
            float *row = vbuf + int64_t(k) * d;
            if (c < cend) row[c] = o.x;
            if (c + 1 < cend) row[c + 1] = o.y;
            if (c + 2 < cend) row[c + 2] = o.z;
            if (c + 3 < cend) row[c + 3] = o.w;
        }
    }
}

}  // namespace dev
}  // namespace tfi
