// Cross tables and component corrections summed directly on the 5th-generation
// tensor cores (tcgen05, kind::tf32), with the accumulator restarted for every
// chunk of 32 source bins.
//
// A direct job evaluates one table at its occupied bins (a call's cross table G at
// its A-bins, Eq. "sumofFFTterms", or a component's correction E_alpha at its
// b-bins, Eq. "stad-E"):
//   val[i] = sum_j f(r_i + r_j + |x_i - x_j|) sum[j]
// over the job's keys (depth r and backbone coordinate x in grid units; x = 0 for
// a one-dimensional correction). It is the f(D) x S product of the dense leaves
// with D(i, j) = r_i + r_j + |x_i - x_j|, so it reuses their scheme: 128-row tiles
// of target bins, chunks of 32 source bins; the f samples split into TF32 hi + lo
// and written to tensor memory by eight producer warps, the bin sums split into
// shared memory, 12 MMAs per chunk issued by a ninth warp into one of three
// accumulator buffers, each chunk's result added in FP32 registers. The bin sums
// of a job are consecutive rows of the bin-sum array, so the B operand loads are
// coalesced. Persistent CTAs each take their own list of jobs (assigned on the host
// longest first to the least-loaded CTA; each list runs largest first) and copy the
// next job's keys in with cp.async while a job runs.
#pragma once

#include "leaf_tc32.cuh"

namespace tfi {
namespace tc {

constexpr int kTab32MinKeys = 64;     // smaller tables stay on the FP32-ALU direct kernel
constexpr int kTab32MaxKeys = 4096;   // as do larger ones (their keys would not fit shared memory)

struct Tab32Layout {
    uint32_t b_off, b_bytes, r_off, x_off, rr_off, rx_off, ftab_off, bar_off, bytes;
};

// b: STAGES x (hi, lo) x NB rows; the job's byte-scaled depths 4 r and coordinates x, and
// the next job's raw keys; fts staged f samples; 2 x STAGES mbarriers.
__host__ __device__ inline Tab32Layout table_tc32_layout(int nb, int max_keys, int fts) {
    Tab32Layout o;
    const int stages = leaf_tc32_stages(nb);
    const uint32_t src = (uint32_t(max_keys + kL32Chunk - 1) / kL32Chunk) * kL32Chunk * 4u;
    o.b_bytes = uint32_t(nb / 8) * kL32SboB;
    o.b_off = 0;
    o.r_off = o.b_off + uint32_t(stages) * 2 * o.b_bytes;
    o.x_off = o.r_off + src;
    o.rr_off = o.x_off + src;
    o.rx_off = o.rr_off + src;
    o.ftab_off = o.rx_off + src;
    o.bar_off = (o.ftab_off + uint32_t(fts) * 4 + 15u) & ~15u;
    o.bytes = o.bar_off + uint32_t(stages) * 16;
    return o;
}

// jobs[q] = (kb, ke, two-dimensional, 0), ke - kb in [1, max_keys]; CTA b takes jobs
// cta_ptr[b] .. cta_ptr[b + 1] - 1
template <int NB, bool FS>
__global__ void __launch_bounds__(kL32Threads, 2) table_tc32_kernel(const int4 *__restrict__ jobs,
                                                                    const int32_t *__restrict__ cta_ptr,
                                                                    const int32_t *__restrict__ key_r,
                                                                    const int32_t *__restrict__ key_x, int d,
                                                                    const float *__restrict__ kbuf,
                                                                    float *__restrict__ vbuf,
                                                                    const float *__restrict__ ftab, int fts,
                                                                    int max_keys, int32_t *__restrict__ err) {
    static_assert(NB == 16 || NB == 32 || NB == 64, "channel block");
    constexpr int STAGES = leaf_tc32_stages(NB);
    static_assert(STAGES * (NB + 2 * kL32Chunk) <= int(kL32Tcols), "tensor-memory columns");
    constexpr uint32_t A_COL = uint32_t(STAGES * NB);
    constexpr int HC = NB / 2;
    extern __shared__ __align__(1024) uint8_t smem[];
    const Tab32Layout lay = table_tc32_layout(NB, max_keys, FS ? fts : 0);
    int32_t *sr4 = reinterpret_cast<int32_t *>(smem + lay.r_off);   // 4 r_j (byte offsets)
    int32_t *sx = reinterpret_cast<int32_t *>(smem + lay.x_off);
    int32_t *rr = reinterpret_cast<int32_t *>(smem + lay.rr_off), *rx = reinterpret_cast<int32_t *>(smem + lay.rx_off);
    float *sf = reinterpret_cast<float *>(smem + lay.ftab_off);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + lay.bar_off);   // full[STAGES], done[STAGES]
    uint64_t *done = full + STAGES;
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
    uint32_t g = 0;     // the CTA's chunk counter (the same sequence in both roles)
    int st = 0;         // its stage, g % STAGES
    uint32_t par = 0;   // the parity of its use of that stage, (g / STAGES) & 1
    bool warm = false;  // g >= STAGES
    const int q0 = cta_ptr[blockIdx.x], q1 = cta_ptr[blockIdx.x + 1];
    auto fetch_keys = [&](int q) {
        if (q >= q1) return;
        const int4 jb = jobs[q];
        for (int j = tid; j < jb.y - jb.x; j += kL32Threads) {
            cp_async4(rr + j, key_r + jb.x + j);
            cp_async4(rx + j, key_x + jb.x + j);
        }
    };
    fetch_keys(q0);

    for (int q = q0; q < q1; ++q) {
        const int4 jb = jobs[q];
        const int kb = jb.x, n = jb.y - jb.x, nc = (n + kL32Chunk - 1) / kL32Chunk;
        const bool two_d = jb.z != 0;
        cp_async_wait_all();
        __syncthreads();
        // past the job's last key: r = x = 0, so an entry reads f at r_i + |x_i| (in range); its
        // bin-sum row is zero
        for (int j = tid; j < nc * kL32Chunk; j += kL32Threads) {
            sr4[j] = j < n ? 4 * rr[j] : 0;
            sx[j] = j < n ? rx[j] : 0;
        }
        __syncthreads();
        fetch_keys(q + 1);
        const int n_tiles = (n + kL32Tile - 1) / kL32Tile;

        if (warp == kL32Producers / 32) {
            // MMA issuer: every chunk of every tile of the job
            if (lane == 0) {
                const uint32_t idesc = idesc_tf32(kL32Tile, NB);
                for (int k = 0; k < n_tiles * nc; ++k, ++g) {
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
            // bin-sum rows of a chunk (channels c0 .. c0 + NB): channel pairs, sources fastest
            constexpr int ITEMS = kL32Chunk * NB / 2;
            constexpr int PER = ITEMS / kL32Producers;
            static_assert(ITEMS % kL32Producers == 0, "items");
            const bool vec = (d % 2) == 0;
            auto load_b = [&](int c, float2 *raw) {
#pragma unroll
                for (int u = 0; u < PER; ++u) {
                    const int qq = tid + u * kL32Producers;
                    const int kk = qq % kL32Chunk, ch = c0 + (qq / kL32Chunk) * 2;
                    const int j = c * kL32Chunk + kk;
                    raw[u] = make_float2(0.f, 0.f);
                    if (j < n && ch < d) {
                        const float *src = kbuf + int64_t(kb + j) * d + ch;
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
                const int ri = tile * kL32Tile + rb * 32 + lane;   // this thread's target bin (job offset)
                const bool row_ok = ri < n;
                const int R4 = (row_ok ? sr4[ri] : 0) + fb;        // 4 r_i + the f samples' base
                const int xi = row_ok ? sx[ri] : 0;
                float2 rawb[PER];
                load_b(0, rawb);
#pragma unroll
                for (int e = 0; e < HC; ++e) acc[e] = 0.f;
                const uint32_t g0 = g;
                auto chunk = [&](int c, auto two_d_tag) -> bool {
                    constexpr bool TWO_D = decltype(two_d_tag)::value;
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
                    // A: f(r_i + r_j + |x_i - x_j|) for this thread's row and sources 16 h .. 16 h + 15
                    const int jb0 = c * kL32Chunk + h * 16;
                    int off[16];
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const int4 r4 = *reinterpret_cast<const int4 *>(sr4 + jb0 + 4 * v);
                        off[4 * v + 0] = R4 + r4.x;
                        off[4 * v + 1] = R4 + r4.y;
                        off[4 * v + 2] = R4 + r4.z;
                        off[4 * v + 3] = R4 + r4.w;
                        if constexpr (TWO_D) {
                            const int4 x4 = *reinterpret_cast<const int4 *>(sx + jb0 + 4 * v);
                            off[4 * v + 0] += 4 * abs(xi - x4.x);
                            off[4 * v + 1] += 4 * abs(xi - x4.y);
                            off[4 * v + 2] += 4 * abs(xi - x4.z);
                            off[4 * v + 3] += 4 * abs(xi - x4.w);
                        }
                    }
                    // A columns of a stage: half h at h * 32: hi of its 16 sources, then their lo
                    uint32_t av[32];
#pragma unroll
                    for (int e = 0; e < 16; ++e) split_tf32_rz(fetch(off[e]), av[e], av[16 + e]);
                    tmem_st32(tmem + lane_base + A_COL + uint32_t(st) * 2 * kL32Chunk + uint32_t(h * 32), av);
                    // B: the chunk's bin-sum rows, transposed (row = channel, K = source), hi and lo
                    uint8_t *Bhi = smem + lay.b_off + uint32_t(st) * 2 * lay.b_bytes, *Blo = Bhi + lay.b_bytes;
#pragma unroll
                    for (int u = 0; u < PER; ++u) {
                        const int qq = tid + u * kL32Producers;
                        const int kk = qq % kL32Chunk, nn = (qq / kL32Chunk) * 2;
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
                if (two_d) {
                    for (int c = 0; c < nc && ok; ++c) ok = chunk(c, std::true_type());
                } else {
                    for (int c = 0; c < nc && ok; ++c) ok = chunk(c, std::false_type());
                }
                // the tile's last min(nc, STAGES) chunks remain (each waited for)
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
                    float *dst = vbuf + int64_t(kb + ri) * d + c0 + h * HC;
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
        // the next job's keys overwrite these
        __syncthreads();
        if (s_abort) break;
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kL32Tcols);
}

}  // namespace tc
}  // namespace tfi
