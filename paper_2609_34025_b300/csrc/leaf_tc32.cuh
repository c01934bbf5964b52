// Dense leaves of FP32 fields on the 5th-generation tensor cores (tcgen05,
// kind::tf32), with the accumulator restarted for every chunk of 32 sources.
//
// A leaf call (|V(S)| <= s0) is summed densely: w_i = sum_{j in S} f(dhat(i, j)) x_j
// (Algorithm 5, base case). In the leaf's preorder, dhat(i, j) = D(i) + D(j) - 2 m(i, j)
// with m(i, j) = min over w in (min(i, j), max(i, j)] of D(parent(w)), the depth of the
// pair's lowest common ancestor, so m(i, j) <= min(D(i), D(j)).
//
// A leaf's targets are taken in tiles of 128 rows (one block of NB channels per CTA); a
// tile's sources are the whole leaf, in chunks of 32 aligned to the leaf's start. Warp w < 8
// holds the targets of row block b = w & 3 (32 rows, itself one 32-source block of the
// leaf) and builds the entries of half h = w >> 2 of every chunk's 32 sources. For a
// chunk c other than the warp's own block the range (i, j] splits at block boundaries:
//   c after b:  m = min(Q(i), M(b, c), P(j)),   Q(i) = min pd over (i, end of b],
//   c before b: m = min(Q(j), M(c, b), P(i)),   P(j) = min pd over [start of j's block, j],
// where M(b, c) is the minimum over the blocks strictly between. With the row carry
// r = min(Q(i), M(b, c), D(i)) (or min(M(c, b), P(i), D(i))) and per-source
// U(j) = D(j) - 2 min(P(j), D(j)) (or with Q(j)):
//   dhat = max(D(j) + D(i) - 2 r, U(j) + D(i)),
// an add and an add-max per entry; clamping by D(i) and D(j) leaves m unchanged and
// keeps every term in range. In the warp's own block m is a running minimum: ascending
// over the sources after i, descending over those before it, each seeded from a warp
// scan of the block's parent distances.
//
// Products: f = fhi + flo with fhi = f rounded toward zero to TF32 (exact) and
// flo = f - fhi (|flo| < 2^-10 |f|, its own TF32 truncation costs < 2^-20 |f|); likewise
// x. D_c = Fhi Xhi + Flo Xhi + Fhi Xlo (the dropped Flo Xlo is below 2^-20 |f x|). The
// f(dhat) operand is written straight into tensor memory (tcgen05.st, one lane per
// target row, which is the layout of an A operand there); the field rows are staged in
// shared memory. Every chunk's 12 MMAs (K = 8 each) start a fresh FP32 accumulator in
// tensor memory (one buffer per pipeline stage); the producer threads read a chunk's
// buffer back when they reuse its stage and add it to FP32 registers, chunk by chunk. A chain over a whole 1024-vertex leaf (384 MMAs into one
// accumulator) measured 6.5e-4 normwise on a slowly decaying kernel; chains of 12
// keep the FP32 bound.
#pragma once

#include <type_traits>

#include "leaf_tc.cuh"

namespace tfi {
namespace tc {

constexpr int kL32Tile = 128;      // target rows per CTA (TMEM lanes)
constexpr int kL32Chunk = 32;      // sources per chunk (4 MMAs of K = 8 per product)
constexpr int kL32MaxChunks = 32;  // leaves of at most 1024 vertices
constexpr int kL32Producers = 256;                 // eight warps build the operands
constexpr int kL32Threads = kL32Producers + 32;    // and one warp issues the MMAs
// B operand (sources across lanes, one channel per store): canonical K-major core
// matrices, padded to 144 B along K so that a warp's 32 sources land in 32 distinct banks.
constexpr uint32_t kL32LboB = 144, kL32SboB = (kL32Chunk / 4) * kL32LboB;

__host__ __device__ constexpr int leaf_tc32_stages(int nb) { return nb == 16 ? 3 : 2; }

// tensor-memory columns: STAGES accumulator buffers of NB, then STAGES A operands of
// 2 x 32 (hi, lo); 256 in all for every NB, so two CTAs fit an SM
constexpr uint32_t kL32Tcols = 256;

__device__ __forceinline__ uint32_t l32_off(int row, int k, uint32_t lbo, uint32_t sbo) {
    return uint32_t(row >> 3) * sbo + uint32_t(k >> 2) * lbo + uint32_t(row & 7) * 16u + uint32_t(k & 3) * 4u;
}

struct Leaf32Layout {
    uint32_t b_off, b_bytes, sd_off, ur_off, ul_off, vtx_off, p_off, q_off, pd_off, raw_off, ftab_off, bar_off, bytes;
};

// b: STAGES x (hi, lo) x NB rows; per-source arrays for max_leaf sources (the parent distances with
// 32 more, read one past a block); the next leaf's raw D, pd and vertex ids (copied in while the
// current leaf runs); fts staged f samples; 2 x STAGES mbarriers.
__host__ __device__ inline Leaf32Layout leaf_tc32_layout(int nb, int max_leaf, int fts) {
    Leaf32Layout o;
    const int stages = leaf_tc32_stages(nb);
    const uint32_t src = (uint32_t(max_leaf + kL32Chunk - 1) / kL32Chunk) * kL32Chunk * 4u;
    o.b_bytes = uint32_t(nb / 8) * kL32SboB;
    o.b_off = 0;
    o.sd_off = o.b_off + uint32_t(stages) * 2 * o.b_bytes;
    o.ur_off = o.sd_off + src;
    o.ul_off = o.ur_off + src;
    o.vtx_off = o.ul_off + src;
    o.p_off = o.vtx_off + src;
    o.q_off = o.p_off + src;
    o.pd_off = o.q_off + src;
    o.raw_off = o.pd_off + src + kL32Chunk * 4;
    o.ftab_off = o.raw_off + 3 * src;
    o.bar_off = (o.ftab_off + uint32_t(fts) * 4 + 15u) & ~15u;
    o.bytes = o.bar_off + uint32_t(stages) * 16;
    return o;
}

__device__ __forceinline__ void split_tf32_rz(float x, uint32_t &hi, uint32_t &lo) {
    hi = __float_as_uint(x) & 0xffffe000u;
    lo = __float_as_uint(x - __uint_as_float(hi));
}

__device__ __forceinline__ float lds_f32(uint32_t addr) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
}

__device__ __forceinline__ void bar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// 32 consecutive 32-bit TMEM columns of this warp's 32 lanes, from registers.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t *r) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]),
        "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),
        "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}

// 4-byte asynchronous copy global -> shared (cp.async), and the wait for all of a thread's copies.
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// D (TMEM) += A (TMEM) x B (shared memory descriptor), kind::tf32.
__device__ __forceinline__ void mma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                            uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc));
}

// Persistent: each CTA takes its own list of leaves, cta_ptr[b] .. cta_ptr[b + 1] - 1 (the host
// assigns them longest first to the least-loaded CTA; each list runs largest first),
// stages a leaf's per-source tables once (its raw inputs copied in with cp.async while
// the previous leaf runs) and runs its 128-row tiles one after another; the f samples are
// staged once per CTA and the tensor memory is held throughout. Warps 0-7 build chunk
// g's operands (g counts the CTA's chunks) in stage g % STAGES and arrive on full[stage];
// one thread of warp 8 waits for it, issues the chunk's 12 MMAs into that stage's
// accumulator buffer and commits them to done[stage]. Before reusing a stage the
// producers wait on done for chunk g - STAGES and, if that chunk belongs to the same
// tile, add its accumulator to their registers; a tile ends by waiting for its last
// chunks and adding their buffers.
template <int NB, bool FS>
__global__ void __launch_bounds__(kL32Threads, 2) leaf_tc32_kernel(const int2 *__restrict__ leaves,
                                                                   const int32_t *__restrict__ cta_ptr,
                                                                   const int32_t *__restrict__ leaf_vtx,
                                                                   const int32_t *__restrict__ leaf_dist,
                                                                   const int32_t *__restrict__ leaf_pdist,
                                                                   const float *__restrict__ F, int d,
                                                                   const float *__restrict__ ftab, int fts,
                                                                   int max_leaf, float *__restrict__ leaf_out,
                                                                   const int32_t *__restrict__ leaf_row,
                                                                   int32_t *__restrict__ err) {
    static_assert(NB == 16 || NB == 32 || NB == 64, "channel block");
    constexpr int STAGES = leaf_tc32_stages(NB);
    static_assert(STAGES * (NB + 2 * kL32Chunk) <= int(kL32Tcols), "tensor-memory columns");
    constexpr uint32_t A_COL = uint32_t(STAGES * NB);   // first A column
    constexpr int HC = NB / 2;   // accumulator columns a producer thread reads back
    constexpr int INF = 0x3fffffff;
    extern __shared__ __align__(1024) uint8_t smem[];
    const Leaf32Layout lay = leaf_tc32_layout(NB, max_leaf, FS ? fts : 0);
    // per-source tables hold byte offsets into the f samples: 4 D(j), 4 U(j)
    int32_t *ssd = reinterpret_cast<int32_t *>(smem + lay.sd_off);
    int32_t *sur = reinterpret_cast<int32_t *>(smem + lay.ur_off);
    int32_t *sul = reinterpret_cast<int32_t *>(smem + lay.ul_off);
    int32_t *svtx = reinterpret_cast<int32_t *>(smem + lay.vtx_off);
    int32_t *sP = reinterpret_cast<int32_t *>(smem + lay.p_off);
    int32_t *sQ = reinterpret_cast<int32_t *>(smem + lay.q_off);
    int32_t *spd = reinterpret_cast<int32_t *>(smem + lay.pd_off);
    const uint32_t src_n = (lay.raw_off - lay.pd_off - kL32Chunk * 4) / 4;   // entries per source array
    int32_t *rdist = reinterpret_cast<int32_t *>(smem + lay.raw_off), *rpd = rdist + src_n, *rvtx = rpd + src_n;
    float *sf = reinterpret_cast<float *>(smem + lay.ftab_off);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + lay.bar_off);   // full[STAGES], done[STAGES]
    uint64_t *done = full + STAGES;
    __shared__ int32_t s_cmin[kL32MaxChunks];
    __shared__ uint32_t s_tmem;
    __shared__ int32_t s_abort;

    const int c0 = blockIdx.y * NB;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tmem_alloc(&s_tmem, kL32Tcols);
    if (tid == kL32Producers) {
        for (int s = 0; s < STAGES; ++s) {
            bar_init(full + s, kL32Producers);
            bar_init(done + s, 1);
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (FS) {
        const int n4 = fts / 4;
        for (int k = tid; k < n4; k += kL32Threads)
            reinterpret_cast<float4 *>(sf)[k] = __ldg(reinterpret_cast<const float4 *>(ftab) + k);
        for (int k = 4 * n4 + tid; k < fts; k += kL32Threads) sf[k] = ftab[k];
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = s_tmem;
    const uint32_t b_base = smem_addr(smem + lay.b_off);
    const int fb = FS ? int(smem_addr(sf)) : 0;
    auto fetch = [&](int off) -> float {
        if constexpr (FS) return lds_f32(uint32_t(off));
        else return __ldg(reinterpret_cast<const float *>(reinterpret_cast<const char *>(ftab) + off));
    };
    uint32_t g = 0;   // the CTA's chunk counter (the same sequence in both roles)
    int st = 0;        // its stage, g % STAGES
    uint32_t par = 0;  // the parity of its use of that stage, (g / STAGES) & 1
    bool warm = false; // g >= STAGES
    // this CTA's leaves, largest first
    const int L0 = cta_ptr[blockIdx.x], L1 = cta_ptr[blockIdx.x + 1];
    // a leaf's raw inputs are copied in asynchronously while the previous leaf runs
    auto fetch_raw = [&](int L) {
        if (L >= L1) return;
        const int2 lf = leaves[L];
        for (int j = tid; j < lf.y - lf.x; j += kL32Threads) {
            cp_async4(rdist + j, leaf_dist + lf.x + j);
            cp_async4(rpd + j, leaf_pdist + lf.x + j);
            cp_async4(rvtx + j, leaf_vtx + lf.x + j);
        }
    };
    fetch_raw(L0);

    for (int L = L0; L < L1; ++L) {
        const int2 lf = leaves[L];
        const int n = lf.y - lf.x, nc = (n + kL32Chunk - 1) / kL32Chunk;
        cp_async_wait_all();
        __syncthreads();
        // per-source tables, one warp per 32-source block: P and Q by warp scans
        for (int c = warp; c < nc; c += kL32Threads / 32) {
            const int j = c * kL32Chunk + lane;
            const bool ok = j < n;
            const int dj = ok ? rdist[j] : 0;
            const int pj = ok ? rpd[j] : INF;
            const int vj = ok ? rvtx[j] : 0;
            int p = pj;   // prefix min over [start, j]
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, p, o);
                if (lane >= o) p = min(p, u);
            }
            int q = __shfl_down_sync(0xffffffffu, pj, 1);   // suffix min over (j, end]
            if (lane == 31) q = INF;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_down_sync(0xffffffffu, q, o);
                if (lane + o < 32) q = min(q, u);
            }
            // past the leaf: D = U = 0, so an entry reads f at D(i) (in range); its field row is zero
            ssd[j] = 4 * dj;
            sur[j] = ok ? 4 * (dj - 2 * min(p, dj)) : 0;
            sul[j] = ok ? 4 * (dj - 2 * min(q, dj)) : 0;
            svtx[j] = vj;
            sP[j] = p;
            sQ[j] = q;
            spd[j] = pj;
            const int cm = __reduce_min_sync(0xffffffffu, pj);
            if (lane == 0) s_cmin[c] = cm;
        }
        if (tid < kL32Chunk) spd[nc * kL32Chunk + tid] = INF;
        __syncthreads();
        fetch_raw(L + 1);
        const int n_tiles = (n + kL32Tile - 1) / kL32Tile;

        if (warp == kL32Producers / 32) {
            // MMA issuer: every chunk of every tile of the leaf
            if (lane == 0) {
                const uint32_t idesc = idesc_tf32(kL32Tile, NB);
                for (int q = 0; q < n_tiles * nc; ++q, ++g) {
                    const int stage = st;
                    if (++st == STAGES) st = 0;
                    const uint32_t ph = par;
                    if (st == 0) par ^= 1u;
                    if (!bar_wait(full + stage, ph)) {
                        atomicExch(err, 1);
                        s_abort = 1;
                        break;
                    }
                    fence_after_sync();
                    const uint32_t abase = tmem + A_COL + uint32_t(stage) * 2 * kL32Chunk;
                    const uint32_t bhi = b_base + uint32_t(stage) * 2 * lay.b_bytes, blo = bhi + lay.b_bytes;
                    const uint32_t dt = tmem + uint32_t(stage * NB);
#pragma unroll
                    for (int ks = 0; ks < kL32Chunk / 8; ++ks) {
                        const uint64_t bh = sdesc(bhi + ks * 2 * kL32LboB, kL32LboB, kL32SboB);
                        const uint64_t bl = sdesc(blo + ks * 2 * kL32LboB, kL32LboB, kL32SboB);
                        const uint32_t ahi = abase + uint32_t((ks >> 1) * 32 + (ks & 1) * 8), alo = ahi + 16;
                        mma_tf32_ts(dt, ahi, bh, idesc, ks > 0 ? 1u : 0u);
                        mma_tf32_ts(dt, alo, bh, idesc, 1u);
                        mma_tf32_ts(dt, ahi, bl, idesc, 1u);
                    }
                    mma_commit(done + stage);
                }
            }
        } else {
            const int rb = warp & 3, h = warp >> 2;
            const uint32_t lane_base = uint32_t(rb * 32) << 16;
            // field rows of a chunk (channels c0 .. c0 + NB): channel pairs, sources fastest
            constexpr int ITEMS = kL32Chunk * NB / 2;
            constexpr int PER = ITEMS / kL32Producers;
            static_assert(ITEMS % kL32Producers == 0, "items");
            const bool vec = (d % 2) == 0 && (reinterpret_cast<uintptr_t>(F) & 7u) == 0;
            auto load_b = [&](int c, float2 *raw) {
#pragma unroll
                for (int u = 0; u < PER; ++u) {
                    const int q = tid + u * kL32Producers;
                    const int kk = q % kL32Chunk, ch = c0 + (q / kL32Chunk) * 2;
                    const int j = c * kL32Chunk + kk;
                    raw[u] = make_float2(0.f, 0.f);
                    if (j < n && ch < d) {
                        const float *src = F + int64_t(svtx[j]) * d + ch;
                        if (vec) {
                            raw[u] = __ldg(reinterpret_cast<const float2 *>(src));
                        } else {
                            raw[u].x = __ldg(src);
                            if (ch + 1 < d) raw[u].y = __ldg(src + 1);
                        }
                    }
                }
            };
            float acc[HC];
            auto read_back = [&](int buf) {
#pragma unroll
                for (int cc = 0; cc < HC; cc += 8) {
                    float v[8];
                    tmem_ld8(tmem + lane_base + uint32_t(buf * NB + h * HC + cc), v);
#pragma unroll
                    for (int e = 0; e < 8; ++e) acc[cc + e] += v[e];
                }
            };
            bool ok = true;
            for (int tile = 0; tile < n_tiles && ok; ++tile) {
                const int t0 = tile * kL32Tile;
                const int bc = t0 / kL32Chunk + rb;           // the warp's row block as a chunk of the leaf
                const int ri = t0 + rb * kL32Chunk + lane;    // this thread's target (leaf offset)
                const bool row_ok = ri < n;
                const int di = row_ok ? ssd[ri] >> 2 : 0;
                const int Pi = row_ok ? sP[ri] : 0, Qi = row_ok ? sQ[ri] : 0;
                const int D4 = 4 * di + fb;
                // the warp's own block: running-minimum seeds from scans of its 32 parent
                // distances (source k of the block has pd[k]); up: min pd over (lane, 16 h - 1]
                // for lanes below this half, down: min pd over [16 h + 16, lane] for lanes above it
                const int *pd = spd + bc * kL32Chunk;
                int seed_up = INF, seed_dn = INF;
                if (bc < nc) {
                    const int pdl = pd[lane];
                    int sfx = __shfl_down_sync(0xffffffffu, pdl, 1);   // min over (lane, 15] in the low half
                    if (lane == 15 || lane == 31) sfx = INF;
#pragma unroll
                    for (int o = 1; o < 16; o <<= 1) {
                        const int u = __shfl_down_sync(0xffffffffu, sfx, o);
                        if ((lane & 15) + o < 16) sfx = min(sfx, u);
                    }
                    int pfx = pdl;                                      // min over [16, lane] in the high half
#pragma unroll
                    for (int o = 1; o < 16; o <<= 1) {
                        const int u = __shfl_up_sync(0xffffffffu, pfx, o);
                        if ((lane & 15) >= o) pfx = min(pfx, u);
                    }
                    if (h == 1 && lane < 16) seed_up = sfx;
                    if (h == 0 && lane >= 16) seed_dn = pfx;
                }
                // M(b, c) for this warp's block b = bc: lane c holds the min over the blocks strictly
                // between, after (mR) or before (mL) b
                int mR, mL;
                {
                    const int cm = lane < nc ? s_cmin[lane] : INF;
                    int v = lane > bc ? cm : INF;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int u = __shfl_up_sync(0xffffffffu, v, o);
                        if (lane >= o) v = min(v, u);
                    }
                    mR = __shfl_up_sync(0xffffffffu, v, 1);
                    if (lane == 0) mR = INF;
                    int w = lane < bc ? cm : INF;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int u = __shfl_down_sync(0xffffffffu, w, o);
                        if (lane + o < 32) w = min(w, u);
                    }
                    mL = __shfl_down_sync(0xffffffffu, w, 1);
                    if (lane == 31) mL = INF;
                }
                float2 rawb[PER];
                load_b(0, rawb);
#pragma unroll
                for (int e = 0; e < HC; ++e) acc[e] = 0.f;
                const uint32_t g0 = g;
                // one chunk; KIND 0: before the warp's block, 1: the block itself, 2: after it
                auto chunk = [&](int c, auto kind_tag) -> bool {
                    constexpr int KIND = decltype(kind_tag)::value;
                    if (warm) {
                        // this stage's operands and accumulator were used by chunk g - STAGES
                        if (!bar_wait(done + st, par ^ 1u)) return false;
                        fence_after_sync();
                        if (c >= STAGES) read_back(st);
                    }
                    float2 cur[PER];
#pragma unroll
                    for (int u = 0; u < PER; ++u) cur[u] = rawb[u];
                    if (c + 1 < nc) load_b(c + 1, rawb);
                    // A: f(dhat) for this thread's row and sources 16 h .. 16 h + 15 of the chunk
                    const int jb = c * kL32Chunk + h * 16;
                    int off[16];
                    if constexpr (KIND != 1) {
                        const int mid = __shfl_sync(0xffffffffu, KIND == 2 ? mR : mL, c);
                        const int r = min(min(KIND == 2 ? Qi : Pi, mid), di);
                        const int A4 = 4 * (di - 2 * r) + fb;
                        const int32_t *U = KIND == 2 ? sur : sul;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int4 s4 = *reinterpret_cast<const int4 *>(ssd + jb + 4 * q);
                            const int4 u4 = *reinterpret_cast<const int4 *>(U + jb + 4 * q);
                            off[4 * q + 0] = max(s4.x + A4, u4.x + D4);
                            off[4 * q + 1] = max(s4.y + A4, u4.y + D4);
                            off[4 * q + 2] = max(s4.z + A4, u4.z + D4);
                            off[4 * q + 3] = max(s4.w + A4, u4.w + D4);
                        }
                    } else {
                        // own block: m(i, j) as running minima over the block's parent distances
                        int m[16];
                        int mu = seed_up;
#pragma unroll
                        for (int e = 0; e < 16; ++e) {            // sources after i, ascending
                            const int k = h * 16 + e;
                            if (k > lane) mu = min(mu, pd[k]);
                            m[e] = mu;
                        }
                        int md = seed_dn;
#pragma unroll
                        for (int e = 15; e >= 0; --e) {           // sources before i, descending
                            const int k = h * 16 + e;
                            if (k < lane) {
                                md = min(md, pd[k + 1]);
                                m[e] = md;
                            }
                        }
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const int k = h * 16 + e, j = c * kL32Chunk + k;
                            const int o = k == lane ? 0
                                        : (!row_ok || j >= n) ? 4 * di
                                                              : 4 * di + ssd[j] - 8 * min(m[e], di);
                            off[e] = o + fb;
                        }
                    }
                    // A columns of a stage: half h at h * 32: hi of its 16 sources, then their lo
                    uint32_t av[32];
#pragma unroll
                    for (int e = 0; e < 16; ++e) split_tf32_rz(fetch(off[e]), av[e], av[16 + e]);
                    tmem_st32(tmem + lane_base + A_COL + uint32_t(st) * 2 * kL32Chunk + uint32_t(h * 32), av);
                    // B: the chunk's field rows, transposed (row = channel, K = source), hi and lo
                    uint8_t *Bhi = smem + lay.b_off + uint32_t(st) * 2 * lay.b_bytes, *Blo = Bhi + lay.b_bytes;
#pragma unroll
                    for (int u = 0; u < PER; ++u) {
                        const int q = tid + u * kL32Producers;
                        const int kk = q % kL32Chunk, nn = (q / kL32Chunk) * 2;
                        uint32_t hb, lb;
                        split_tf32_rz(cur[u].x, hb, lb);
                        *reinterpret_cast<uint32_t *>(Bhi + l32_off(nn, kk, kL32LboB, kL32SboB)) = hb;
                        *reinterpret_cast<uint32_t *>(Blo + l32_off(nn, kk, kL32LboB, kL32SboB)) = lb;
                        split_tf32_rz(cur[u].y, hb, lb);
                        *reinterpret_cast<uint32_t *>(Bhi + l32_off(nn + 1, kk, kL32LboB, kL32SboB)) = hb;
                        *reinterpret_cast<uint32_t *>(Blo + l32_off(nn + 1, kk, kL32LboB, kL32SboB)) = lb;
                    }
                    // operands visible to the tensor cores; the tensor-memory stores and read-back
                    // ordered before the MMAs that follow the arrival
                    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                    fence_async_smem();
                    fence_before_sync();
                    bar_arrive(full + st);
                    ++g;
                    if (++st == STAGES) {
                        st = 0;
                        par ^= 1u;
                        warm = true;
                    }
                    return true;
                };
                // the chunks before the warp's block, the block, the chunks after it (warp-uniform code)
                for (int c = 0; c < min(bc, nc) && ok; ++c) ok = chunk(c, std::integral_constant<int, 0>());
                if (ok && bc < nc) ok = chunk(bc, std::integral_constant<int, 1>());
                for (int c = bc + 1; c < nc && ok; ++c) ok = chunk(c, std::integral_constant<int, 2>());
                // the tile's last min(nc, STAGES) chunks remain (each committed by the thread
                // that issued it, so each is waited for)
                for (int c = max(0, nc - STAGES); c < nc && ok; ++c) {
                    const uint32_t gc = g0 + uint32_t(c);
                    if (bar_wait(done + int(gc % STAGES), (gc / STAGES) & 1u)) {
                        fence_after_sync();
                        read_back(int(gc % STAGES));
                    } else {
                        ok = false;
                    }
                }
                if (ok && row_ok) {
                    float *dst = leaf_out + int64_t(leaf_row[lf.x + ri]) * d + c0 + h * HC;
#pragma unroll
                    for (int e = 0; e < HC; ++e)
                        if (c0 + h * HC + e < d) dst[e] = acc[e];
                }
            }
            if (!ok) {
                atomicExch(err, 1);
                s_abort = 1;
            }
        }
        // the next leaf's tables overwrite these
        __syncthreads();
        if (s_abort) break;
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kL32Tcols);
}

}  // namespace tc
}  // namespace tfi
