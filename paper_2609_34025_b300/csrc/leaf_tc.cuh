// Dense leaves on the 5th-generation tensor cores (tcgen05, kind::tf32).
//
// A leaf call (|V(S)| <= s0) is summed densely: w_u = sum_{v in S} f(dhat(u, v)) x_v.
// In the leaf's preorder, dhat(i, j) = D(i) + D(j) - 2 m(i, j) with
// m(i, j) = min over w in (min(i, j), max(i, j)] of D(parent(w)). Small leaves
// are packed into groups; a pair from two different leaves of a group is 0.
//
// One CTA of 256 threads per (tile of 128 target rows of a group, block of NB
// channels). The product out[i][c] = sum_j M[i][j] F[j][c] runs over chunks of
// 32 sources: M = 128 x 32 generated in shared memory, F chunk = NB x 32 staged
// from the field rows, D = 128 x NB FP32 accumulators in tensor memory. Every
// pair of a chunk is independent:
//   * diagonal chunks (sources inside the tile's own 128 rows): m(i, j) from a
//     sparse table over the tile's 128 parent distances;
//   * chunks to the right (sources after the tile, visited in ascending order):
//     m(i, j) = min(R_i, P[j]) with the chunk prefix minimum P and the row carry
//     R_i = min over (i, chunk start), updated after each chunk;
//   * chunks to the left (sources before the tile, descending order):
//     m(i, j) = min(Q[j], C_i) with the chunk suffix minimum Q[j] over
//     (j, chunk end] and the row carry C_i = min over (chunk end, i].
// Operands are TF32 hi / lo splits (x = hi + lo, |x - hi - lo| <= 2^-22 |x|):
// D = Mhi Fhi + Mlo Fhi + Mhi Flo for FP32 fields; BF16 fields are exact in
// TF32, so D = Mhi F + Mlo F. Two operand stages: chunk k + 1 is generated
// while the MMAs of chunk k run.
#pragma once

#include "hankel_tc.cuh"

namespace tfi {
namespace tc {

constexpr int kLeafTile = 128;     // target rows per CTA (TMEM lanes)
constexpr int kLeafChunk = 32;     // sources per chunk (4 MMAs of K = 8)
constexpr int kLeafSrcMax = 1024;  // largest source range of a tile (largest leaf or group)
// Operand tiles use the canonical K-major layout without swizzle, with the core
// matrices along K padded to 144 B apart (LBO) instead of packed at 128 B: a
// warp storing one K column of 32 sources then touches 32 distinct banks.
constexpr uint32_t kLeafLbo = 144;
constexpr uint32_t kLeafSbo = (kLeafChunk / 4) * kLeafLbo;  // bytes between 8-row core-matrix groups

__device__ __forceinline__ uint32_t leaf_off(int row, int k) {
    return uint32_t(row >> 3) * kLeafSbo + uint32_t(k >> 2) * kLeafLbo + uint32_t(row & 7) * 16u + uint32_t(k & 3) * 4u;
}

struct LeafTile {
    int32_t gb, ge;   // the group's range in leaf order
    int32_t i0;       // first target row of the tile (absolute)
    int32_t pad;
};

struct LeafTcLayout {
    uint32_t a_off, b_off, b_bytes, dist_off, pd_off, vtx_off, st_off, pq_off, ftab_off, bar_off, bytes;
};

// a: 2 stages x (hi, lo) x 128 rows; b: 2 stages x (hi[, lo]) x NB rows; kLeafSbo per 8 rows.
__host__ __device__ inline LeafTcLayout leaf_tc_layout(int nb, bool split_b, int ftab_smem) {
    LeafTcLayout o;
    const uint32_t a_tile = uint32_t(kLeafTile / 8) * kLeafSbo;
    o.b_bytes = uint32_t(nb / 8) * kLeafSbo;
    o.a_off = 0;
    o.b_off = 4 * a_tile;
    o.dist_off = o.b_off + 2 * (split_b ? 2 : 1) * o.b_bytes;
    o.pd_off = o.dist_off + kLeafSrcMax * 4;
    o.vtx_off = o.pd_off + kLeafSrcMax * 4;
    o.st_off = o.vtx_off + kLeafSrcMax * 4;           // 7 levels x 128
    o.pq_off = o.st_off + 7 * kLeafTile * 4;          // 32 prefix / suffix minima
    o.ftab_off = o.pq_off + kLeafChunk * 4;
    o.bar_off = (o.ftab_off + uint32_t(ftab_smem) * 4 + 15u) & ~15u;
    o.bytes = o.bar_off + 32;
    return o;
}

// 8 consecutive 32-bit TMEM columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

template <typename T>
__device__ __forceinline__ float leaf_ld(const T *p);
template <>
__device__ __forceinline__ float leaf_ld<float>(const float *p) { return *p; }
template <>
__device__ __forceinline__ float leaf_ld<__nv_bfloat16>(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

template <typename T, int NB>
__global__ void __launch_bounds__(256) leaf_tc_kernel(const LeafTile *__restrict__ tiles,
                                                      const int32_t *__restrict__ leaf_vtx,
                                                      const int32_t *__restrict__ leaf_dist,
                                                      const int32_t *__restrict__ leaf_pdist,
                                                      const int32_t *__restrict__ leaf_lo,
                                                      const int32_t *__restrict__ leaf_hi, const T *__restrict__ F,
                                                      int d, const float *__restrict__ ftab, int ftab_smem,
                                                      float *__restrict__ leaf_out,
                                                      const int32_t *__restrict__ leaf_row, int32_t *__restrict__ err) {
    constexpr bool F32 = sizeof(T) == 4;
    constexpr int NSPLIT = F32 ? 2 : 1;
    constexpr uint32_t TCOLS = NB <= 32 ? 32u : uint32_t(NB);
    constexpr uint32_t A_TILE = uint32_t(kLeafTile / 8) * kLeafSbo;
    constexpr int INF = 0x7fffffff;
    extern __shared__ __align__(1024) uint8_t smem[];
    const LeafTcLayout lay = leaf_tc_layout(NB, F32, ftab_smem);
    int32_t *sdist = reinterpret_cast<int32_t *>(smem + lay.dist_off);
    int32_t *spd = reinterpret_cast<int32_t *>(smem + lay.pd_off);
    int32_t *svtx = reinterpret_cast<int32_t *>(smem + lay.vtx_off);
    int32_t *st = reinterpret_cast<int32_t *>(smem + lay.st_off);
    int32_t *pq = reinterpret_cast<int32_t *>(smem + lay.pq_off);
    float *sf = reinterpret_cast<float *>(smem + lay.ftab_off);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + lay.bar_off);  // bar[0], bar[1]
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bar + 2);

    const LeafTile tl = tiles[blockIdx.x];
    const int c0 = blockIdx.y * NB;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = tid & (kLeafTile - 1), half = tid >> 7;
    const int i = tl.i0 + row;                        // this thread's target (absolute)
    const bool row_ok = i < tl.ge;
    const int last = min(tl.i0 + kLeafTile, tl.ge) - 1;
    const int s_lo = leaf_lo[tl.i0], s_hi = leaf_hi[last];   // the tile's sources [s_lo, s_hi)
    const int lo_i = row_ok ? leaf_lo[i] : 0, hi_i = row_ok ? leaf_hi[i] : 0;

    if (warp == 0) tmem_alloc(tmem_holder, TCOLS);
    if (tid == 0) {
        bar_init(bar, 1);
        bar_init(bar + 1, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int j = s_lo + tid; j < s_hi; j += 256) {
        sdist[j - s_lo] = leaf_dist[j];
        spd[j - s_lo] = leaf_pdist[j];
        svtx[j - s_lo] = leaf_vtx[j];
    }
    for (int k = tid; k < ftab_smem; k += 256) sf[k] = ftab[k];
    __syncthreads();
    // sparse table over the tile's parent distances: st[l][x] = min pd[i0 + x .. i0 + x + 2^l - 1]
    for (int x = tid; x < kLeafTile; x += 256) {
        const int j = tl.i0 + x;
        st[x] = j < s_hi ? spd[j - s_lo] : INF;
    }
    __syncthreads();
    for (int l = 1; l < 7; ++l) {
        for (int x = tid; x < kLeafTile; x += 256) {
            const int y = x + (1 << (l - 1));
            st[l * kLeafTile + x] = min(st[(l - 1) * kLeafTile + x], y < kLeafTile ? st[(l - 1) * kLeafTile + y] : INF);
        }
        __syncthreads();
    }
    const float *fsrc = ftab_smem > 0 ? sf : ftab;
    auto rmq = [&](int a, int b) {  // min pd over tile offsets [a, b], 0 <= a <= b < 128
        const int l = 31 - __clz(b - a + 1);
        return min(st[l * kLeafTile + a], st[l * kLeafTile + b - (1 << l) + 1]);
    };
    const int ri = row;
    const int di = row_ok ? sdist[i - s_lo] : 0;
    // carries at the tile edges: R = min pd over (i, i0 + 127], C = min pd over (i0, i]
    int carry_r = ri < kLeafTile - 1 ? rmq(ri + 1, kLeafTile - 1) : INF;
    int carry_c = ri > 0 ? rmq(1, ri) : INF;

    const int tile_end = min(tl.i0 + kLeafTile, s_hi);
    const int n_diag = (tile_end - tl.i0 + kLeafChunk - 1) / kLeafChunk;
    const int n_right = (s_hi - tile_end + kLeafChunk - 1) / kLeafChunk;
    const int n_left = (tl.i0 - s_lo + kLeafChunk - 1) / kLeafChunk;
    const int n_chunks = n_diag + n_right + n_left;
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_holder;
    const uint32_t idesc = idesc_tf32(kLeafTile, NB);
    bool ok = true;
    for (int ch = 0; ch < n_chunks; ++ch) {
        const int stage = ch & 1;
        // kind: 0 diagonal, 1 right, 2 left; j0 = first source of the chunk
        int kind, j0;
        if (ch < n_diag) {
            kind = 0;
            j0 = tl.i0 + ch * kLeafChunk;
        } else if (ch < n_diag + n_right) {
            kind = 1;
            j0 = tile_end + (ch - n_diag) * kLeafChunk;
        } else {
            kind = 2;
            j0 = tl.i0 - (ch - n_diag - n_right + 1) * kLeafChunk;
        }
        // this stage's operands were read by the MMAs of chunk ch - 2
        if (ch >= 2) {
            const bool done = bar_wait(bar + stage, uint32_t(((ch - 2) >> 1) & 1));
            ok = __syncthreads_and(done ? 1 : 0) != 0;
            fence_after_sync();
            if (!ok) break;
        }
        // chunk prefix (right) or suffix (left) minima of the parent distances
        if (kind != 0 && warp == 0) {
            const int lane = tid & 31;
            if (kind == 1) {
                const int j = j0 + lane;
                int v = j < s_hi ? spd[j - s_lo] : INF;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int u = __shfl_up_sync(0xffffffffu, v, o);
                    if (lane >= o) v = min(v, u);
                }
                pq[lane] = v;                                  // min pd[j0 .. j0 + lane]
            } else {
                const int j = j0 + lane + 1;                   // (j0 + lane, j0 + 32]
                int v = (j >= s_lo && j < s_hi) ? spd[j - s_lo] : INF;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int u = __shfl_down_sync(0xffffffffu, v, o);
                    if (lane + o < 32) v = min(v, u);
                }
                pq[lane] = v;                                  // min pd[j0 + lane + 1 .. j0 + 32]
            }
        }
        __syncthreads();
        // A: f(dhat) for this thread's row and 16 sources, split hi / lo
        uint8_t *Ahi = smem + lay.a_off + uint32_t(stage) * 2 * A_TILE, *Alo = Ahi + A_TILE;
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            uint4 h, lo;
            uint32_t *hp = &h.x, *lp = &lo.x;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int kk = half * 16 + g * 4 + e;
                const int j = j0 + kk;
                float f = 0.f;
                if (row_ok && j >= lo_i && j < hi_i) {
                    int m;
                    if (kind == 0) {
                        const int rj = j - tl.i0;
                        m = rj == ri ? INF : (rj > ri ? rmq(ri + 1, rj) : rmq(rj + 1, ri));
                    } else if (kind == 1) {
                        m = min(carry_r, pq[kk]);
                    } else {
                        m = min(pq[kk], carry_c);
                    }
                    f = j == i ? fsrc[0] : fsrc[di + sdist[j - s_lo] - 2 * m];
                }
                split_tf32(f, hp[e], lp[e]);
            }
            *reinterpret_cast<uint4 *>(Ahi + leaf_off(row, half * 16 + g * 4)) = h;
            *reinterpret_cast<uint4 *>(Alo + leaf_off(row, half * 16 + g * 4)) = lo;
        }
        if (kind == 1) carry_r = min(carry_r, pq[kLeafChunk - 1]);
        if (kind == 2) carry_c = min(carry_c, pq[0]);
        // B: field rows of the chunk's sources, channels c0 .. c0 + NB (hi [, lo]). Each item is
        // 16 bytes of one source row (VE channels); sources vary fastest across threads so that
        // the transposed stores of a warp fall in distinct banks. All loads are issued first.
        uint8_t *Bhi = smem + lay.b_off + uint32_t(stage) * NSPLIT * lay.b_bytes, *Blo = Bhi + lay.b_bytes;
        {
            constexpr int VE = 16 / int(sizeof(T));              // channels per 16-byte item
            constexpr int ITEMS = kLeafChunk * NB / VE;
            constexpr int PER = (ITEMS + 255) / 256;
            const bool vec = (d % VE) == 0 && (reinterpret_cast<uintptr_t>(F) & 15u) == 0;
            uint4 raw[PER];
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const int q = tid + u * 256;
                const int kk = q % kLeafChunk, n = (q / kLeafChunk) * VE;
                const int j = j0 + kk, c = c0 + n;
                raw[u] = make_uint4(0u, 0u, 0u, 0u);
                if (q < ITEMS && j >= s_lo && j < s_hi && c < d) {
                    const T *src = F + int64_t(svtx[j - s_lo]) * d + c;
                    if (vec) {
                        raw[u] = __ldg(reinterpret_cast<const uint4 *>(src));
                    } else {
                        T tmp[VE];
#pragma unroll
                        for (int e = 0; e < VE; ++e) tmp[e] = (c + e < d) ? src[e] : T(0.f);
                        raw[u] = *reinterpret_cast<const uint4 *>(tmp);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const int q = tid + u * 256;
                if (q >= ITEMS) break;
                const int kk = q % kLeafChunk, n = (q / kLeafChunk) * VE;
                const T *vals = reinterpret_cast<const T *>(&raw[u]);
#pragma unroll
                for (int e = 0; e < VE; ++e) {
                    uint32_t h, lo;
                    split_tf32(leaf_ld<T>(vals + e), h, lo);
                    *reinterpret_cast<uint32_t *>(Bhi + leaf_off(n + e, kk)) = h;
                    if (F32) *reinterpret_cast<uint32_t *>(Blo + leaf_off(n + e, kk)) = lo;
                }
            }
        }
        fence_async_smem();
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
        if (tid == 0) {
#pragma unroll
            for (int ks = 0; ks < kLeafChunk / 8; ++ks) {
                const uint32_t acc = (ch > 0 || ks > 0) ? 1u : 0u;
                const uint32_t ko = uint32_t(ks) * 2 * kLeafLbo;  // K = 8: two core matrices along K
                const uint64_t ah = sdesc(smem_addr(Ahi) + ko, kLeafLbo, kLeafSbo);
                const uint64_t al = sdesc(smem_addr(Alo) + ko, kLeafLbo, kLeafSbo);
                const uint64_t bh = sdesc(smem_addr(Bhi) + ko, kLeafLbo, kLeafSbo);
                mma_tf32(tmem, ah, bh, idesc, acc);
                mma_tf32(tmem, al, bh, idesc, 1u);
                if (F32) {
                    const uint64_t bl = sdesc(smem_addr(Blo) + ko, kLeafLbo, kLeafSbo);
                    mma_tf32(tmem, ah, bl, idesc, 1u);
                }
            }
            mma_commit(bar + stage);
        }
    }
    // the last commit covers every MMA issued before it
    if (ok && n_chunks > 0) {
        const int lc = n_chunks - 1;
        const bool done = bar_wait(bar + (lc & 1), uint32_t((lc >> 1) & 1));
        ok = __syncthreads_and(done ? 1 : 0) != 0;
        fence_after_sync();
    }
    if (!ok && tid == 0) atomicExch(err, 1);
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31; the two warp quarters split the columns
    if (ok && n_chunks > 0) {
        const uint32_t lane_base = uint32_t((warp & 3) * 32) << 16;
        const int trow = tl.i0 + (warp & 3) * 32 + (tid & 31);
        const bool wr = trow < tl.ge;
        float *dst = wr ? leaf_out + int64_t(leaf_row[trow]) * d : nullptr;
        constexpr int HALF_COLS = NB >= 32 ? NB / 2 : NB;
        const int cb = NB >= 32 ? half * HALF_COLS : 0;
        if (NB >= 32 || half == 0) {
#pragma unroll 1
            for (int cc = 0; cc < HALF_COLS; cc += 8) {
                float v[8];
                tmem_ld8(tmem + lane_base + uint32_t(cb + cc), v);
                if (wr) {
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int c = c0 + cb + cc + e;
                        if (c < d) dst[c] = v[e];
                    }
                }
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TCOLS);
}

}  // namespace tc
}  // namespace tfi
