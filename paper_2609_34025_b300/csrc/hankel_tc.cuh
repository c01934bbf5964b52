// Cross tables by a Hankel-matrix product on the 5th-generation tensor cores.
//
// Attention-width evaluation of Eq. "sumofFFTterms" (appendix on the cross term
// at attention width). With l = q + |s - t| the kernel argument is l + r, so
//     B[l, t] = sum_r f(l + r) A_r[t]         (l = 0 .. H + L)
// is one product with the Hankel matrix Fh[l][r] = f(l + r), and
//     G_q[s] = sum_t B[q + |s - t|, t]
//            = sum_{t <= s} B[q + s - t, t] + sum_{t >= s} B[q + t - s, t] - B[q, s].
// The left sum runs along the antidiagonal l + t = q + s and the right sum along
// the diagonal l - t = q - s, so both are prefix sums over t.
//
// One CTA of 128 threads per (job, block of 128 channels). The MMA is
// D[c][l] = sum_r A_t[c][r] Fh[l][r]: M = 128 channels (one TMEM lane per
// channel), N = the table's rows l, K = depths r, so thread c reads B[., t] for
// its own channel from its TMEM lane and runs both scans in shared memory
// without exchanging data with other threads. Columns t are visited in
// ascending order; at t = s, for every occupied bin (q, s):
//     out = L_q[s] - B[q, s] - (sum_{t < s} B[q + t - s, t])
// and after the last column the diagonal totals sum_t B[q + t - s, t] are added,
// which turns the subtracted prefix into the suffix sum_{t >= s}. Columns
// without occupied bins contribute B[., t] = 0 and are skipped.
//
// Operands are TF32 hi / lo splits of the FP32 values (f samples and bin sums),
// x = hi + lo with |x - hi - lo| <= 2^-22 |x|, and the MMA is kind::tf32:
// D = Ahi Fhi + Ahi Flo + Alo Fhi with FP32 accumulation in tensor memory
// (relative error ~2^-21 per product, on a par with FP32 arithmetic). The
// shared-memory operands use the canonical K-major layout without swizzle:
// 8-row x 16-byte core matrices (4 TF32 values along K), LBO = 128 B between
// core matrices along K, SBO = KT x 32 B between 8-row groups.
#pragma once

#include "dense_tc.cuh"
#include "hankel_layout.hpp"

namespace tfi {
namespace tc {

struct HankelItem {
    int32_t kb, ke;  // the job's key range
    int32_t c0;      // first channel of the block
    int32_t H;       // largest depth among the job's bins (grid units)
    int32_t L;       // largest coordinate among the job's bins (grid units)
    int32_t pad[3];
};

// Instruction descriptor, kind::tf32: D = F32, A = B = TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(m >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// x = hi + lo in TF32
__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo) {
    hi = to_tf32(x);
    lo = to_tf32(x - __uint_as_float(hi));
}

// Byte offset of element (row, k) in a K-major TF32 operand tile.
__device__ __forceinline__ uint32_t kmajor_off_tf32(int row, int k, uint32_t sbo) {
    return uint32_t(row >> 3) * sbo + uint32_t(k >> 2) * 128u + uint32_t(row & 7) * 16u + uint32_t(k & 3) * 4u;
}

// Writes val = G at every occupied bin of the item's job for channels c0 .. c0+127.
__global__ void __launch_bounds__(128) hankel_kernel(const HankelItem *__restrict__ items,
                                                     const int32_t *__restrict__ key_r,
                                                     const int32_t *__restrict__ key_x, int d,
                                                     const float *__restrict__ kbuf, float *__restrict__ vbuf,
                                                     const float *__restrict__ ftab, int32_t *__restrict__ err) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const HankelItem it = items[blockIdx.x];
    const int H = it.H, Lx = it.L;
    const HankelLayout lay = hankel_layout(H, Lx);
    const int S = lay.S, NP = lay.NP, KT = lay.KT, W = lay.W;
    const uint32_t sbo = lay.sbo;
    uint8_t *Ahi = smem, *Alo = smem + lay.a_bytes;
    uint8_t *Fhi = smem + lay.f_off, *Flo = Fhi + lay.f_bytes;
    int32_t *map = reinterpret_cast<int32_t *>(smem + lay.map_off);
    int32_t *col = reinterpret_cast<int32_t *>(smem + lay.col_off);
    float *accL = reinterpret_cast<float *>(smem + lay.acc_off);
    float *accD = accL + S * 128;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + lay.bar_off);
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bar + 1);
    const uint32_t tcols = hankel_tmem_cols(NP);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int kb = it.kb, ke = it.ke;
    if (warp == 0) tmem_alloc(tmem_holder, tcols);
    if (tid == 0) {
        bar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = tid; i < (H + 1) * W; i += 128) map[i] = -1;
    for (int i = tid; i < W; i += 128) col[i] = 0;
    if (Lx > 0)
        for (int i = tid; i < 2 * S * 128; i += 128) accL[i] = 0.f;
    // Fh operand: row l, depth r: f(l + r) for l <= H + L, r <= H (0 in the padding)
    for (int seg = tid; seg < NP * (KT / 4); seg += 128) {
        const int l = seg / (KT / 4), g = seg % (KT / 4);
        uint4 h, lo;
        uint32_t *hp = &h.x, *lp = &lo.x;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int r = g * 4 + e;
            const float f = (l < S && r <= H) ? __ldg(ftab + l + r) : 0.f;
            split_tf32(f, hp[e], lp[e]);
        }
        *reinterpret_cast<uint4 *>(Fhi + kmajor_off_tf32(l, g * 4, sbo)) = h;
        *reinterpret_cast<uint4 *>(Flo + kmajor_off_tf32(l, g * 4, sbo)) = lo;
    }
    __syncthreads();
    for (int k = kb + tid; k < ke; k += 128) {
        const int r = key_r[k], x = key_x[k];
        map[r * W + x] = k;
        col[x] = 1;
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_holder;
    const uint32_t lane_base = uint32_t(warp * 32) << 16;
    const int c = it.c0 + tid;
    const bool cok = c < d;
    const uint32_t idesc = idesc_tf32(128, NP);
    bool ok = true;
    uint32_t phase = 0;
    for (int t = 0; t < W; ++t) {
        if (!col[t]) continue;  // CTA-uniform
        // A_t operand: row = this thread's channel, K = depth r
        for (int g = 0; g < KT / 4; ++g) {
            uint4 h, lo;
            uint32_t *hp = &h.x, *lp = &lo.x;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int r = g * 4 + e;
                const int k = r <= H ? map[r * W + t] : -1;
                const float v = (k >= 0 && cok) ? kbuf[int64_t(k) * d + c] : 0.f;
                split_tf32(v, hp[e], lp[e]);
            }
            *reinterpret_cast<uint4 *>(Ahi + kmajor_off_tf32(tid, g * 4, sbo)) = h;
            *reinterpret_cast<uint4 *>(Alo + kmajor_off_tf32(tid, g * 4, sbo)) = lo;
        }
        fence_async_smem();
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
        if (tid == 0) {
            for (int ks = 0; ks < KT / 8; ++ks) {
                const uint64_t ah = sdesc(smem_addr(Ahi) + ks * 256, 128, sbo);
                const uint64_t al = sdesc(smem_addr(Alo) + ks * 256, 128, sbo);
                const uint64_t fh = sdesc(smem_addr(Fhi) + ks * 256, 128, sbo);
                const uint64_t fl = sdesc(smem_addr(Flo) + ks * 256, 128, sbo);
                mma_tf32(tmem, ah, fh, idesc, ks > 0 ? 1u : 0u);
                mma_tf32(tmem, ah, fl, idesc, 1u);
                mma_tf32(tmem, al, fh, idesc, 1u);
            }
            mma_commit(bar);
        }
        const bool done = bar_wait(bar, phase);
        phase ^= 1u;
        ok = __syncthreads_and(done ? 1 : 0) != 0;  // CTA-uniform
        fence_after_sync();
        if (!ok) break;
        // epilogue for column t: this thread's channel, rows l = 0 .. S-1
        for (int l0 = 0; l0 < S; l0 += 16) {
            float v[16];
            tmem_ld16(tmem + lane_base + uint32_t(l0), v);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int l = l0 + i;
                if (l >= S) break;
                const float b = v[i];
                float lv = b, dv = 0.f;
                if (Lx > 0) {
                    const int iL = l + t, iD = l - t + Lx;
                    if (iL < S) {
                        lv = accL[iL * 128 + tid] + b;
                        accL[iL * 128 + tid] = lv;
                    }
                    if (iD < S) {
                        dv = accD[iD * 128 + tid];
                        accD[iD * 128 + tid] = dv + b;
                    }
                }
                if (l <= H) {
                    const int k = map[l * W + t];
                    if (k >= 0 && cok) vbuf[int64_t(k) * d + c] = Lx > 0 ? lv - b - dv : b;
                }
            }
        }
        // the next column's MMA overwrites the accumulator and reads A again
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
    }
    if (ok && Lx > 0 && cok) {
        // add the diagonal totals: -prefix_{t < s} + total = suffix_{t >= s}
        for (int k = kb; k < ke; ++k) {
            const int iD = key_r[k] - key_x[k] + Lx;
            vbuf[int64_t(k) * d + c] += accD[iD * 128 + tid];
        }
    }
    if (!ok && tid == 0) atomicExch(err, 1);
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, tcols);
}

}  // namespace tc
}  // namespace tfi
