// Dense f(D) x F on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// The plain definition (Eq. "integration"), evaluated densely per tree: for
// each tree, out[i] = sum_j f(dhat(i, j)) F[j] over its vertices. This is the
// dense comparison path ("dense evaluation materialises M = f(D) and applies
// it", runtime protocol of the attention appendix) and the evaluator for small
// trees with many channels. M is never stored: each CTA generates a 128 x 64
// tile of f(D) in shared memory from root distances and a sparse-table range
// minimum over the tree's preorder:
//     dhat(i, j) = D(i) + D(j) - 2 min_{w in (i, j]} D(parent(w))   (i < j)
// splits it into BF16 hi + lo, and multiplies it with a BF16 tile of F by
// tcgen05.mma (kind::f16, FP32 accumulators in tensor memory). FP32 fields are
// split too: out = Mhi Fhi + Mhi Flo + Mlo Fhi (relative error ~2^-16); BF16
// fields: out = Mhi F + Mlo F.
//
// Shared-memory operands use the canonical K-major layout without swizzle:
// 8-row x 16-byte core matrices, LBO = 128 B between core matrices along K,
// SBO = 1024 B between core matrices along M (or N). Every address an MMA can
// form lies inside its own operand tile.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace tfi {
namespace tc {

constexpr int kTileM = 128;   // targets per CTA (TMEM lanes)
constexpr int kTileK = 64;    // sources per chunk (4 MMAs of K = 16)
constexpr uint32_t kSpinLimit = 1u << 26;

struct DenseItem {
    int32_t t0;      // first target of the tile (preorder index)
    int32_t tree;    // tree index
    int32_t c0;      // first channel of the chunk
    int32_t pad;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start, leading / stride byte offsets, the
// fixed version field of sm_100-class descriptors, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = uint64_t((saddr >> 4) & 0x3FFFu);
    d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
    d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
    d |= uint64_t(1) << 46;
    return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void bar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Bounded wait on an mbarrier phase: at most `limit` polls (backing off with a short
// sleep after the first 64); returns false if it gave up.
__device__ __forceinline__ bool bar_wait_n(uint64_t *bar, uint32_t parity, uint32_t limit) {
    const uint32_t a = smem_addr(bar);
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (it > 64) __nanosleep(64);
    }
    return false;
}

// The wait every tensor-core kernel uses on its MMA-completion mbarrier.
__device__ __forceinline__ bool bar_wait(uint64_t *bar, uint32_t parity) { return bar_wait_n(bar, parity, kSpinLimit); }

// Failure-detection self-test: one thread initialises an mbarrier for one arrival,
// optionally arrives on it, then waits for its first phase with at most `limit` polls
// through the same bounded wait as the tensor-core kernels. With no arrival nothing can
// complete the phase, so the wait runs out and the kernel records that in *err and
// returns. No MMA is issued and no tensor memory is allocated.
__global__ void bounded_wait_probe(int arrive, uint32_t limit, int32_t *err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    bar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&bar)) : "memory");
    if (!bar_wait_n(&bar, 0, limit)) *err = 1;
}

__device__ __forceinline__ void tmem_alloc(uint32_t *holder, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(holder)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive 32-bit TMEM columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (row, k) in a K-major, no-swizzle operand tile with
// 64 elements of K per row (8 core matrices of 128 B along K).
__device__ __forceinline__ uint32_t kmajor_off(int row, int k) {
    return uint32_t((row >> 3) * 1024 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

template <typename T>
__device__ __forceinline__ float load_f(const T *p);
template <>
__device__ __forceinline__ float load_f<float>(const float *p) { return *p; }
template <>
__device__ __forceinline__ float load_f<__nv_bfloat16>(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

// One CTA of 128 threads per (tree, 128-target tile, channel chunk of NC).
// F32 fields: NC = 16 (B = [Fhi | Flo], 32 rows). BF16 fields: NC = 64.
template <typename T, int NC>
__global__ void __launch_bounds__(128) dense_tc_kernel(const DenseItem *__restrict__ items,
                                                       const int32_t *__restrict__ tree_ptr,
                                                       const int32_t *__restrict__ vtx, const int32_t *__restrict__ dist,
                                                       const int32_t *__restrict__ st, int64_t n_pre, int levels,
                                                       const float *__restrict__ ftab, const T *__restrict__ F, int d,
                                                       T *__restrict__ out, int32_t *__restrict__ err) {
    constexpr bool F32 = sizeof(T) == 4;
    constexpr int NB = F32 ? 2 * NC : NC;              // rows of B
    constexpr int N1 = NB;                             // MMA 1: Mhi x B
    constexpr int N2 = NC;                             // MMA 2: Mlo x Fhi (first NC rows of B)
    constexpr uint32_t TCOLS = (N1 + N2) <= 32 ? 32 : (N1 + N2) <= 64 ? 64 : (N1 + N2) <= 128 ? 128 : 256;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *Ahi = smem;                               // 128 x 64 bf16 = 16 KB
    uint8_t *Alo = smem + 16384;                       // 16 KB
    uint8_t *B = smem + 32768;                         // NB x 64 bf16
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 32768 + NB * 128);
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bar + 1);

    const DenseItem it = items[blockIdx.x];
    const int tb = tree_ptr[it.tree], te = tree_ptr[it.tree + 1];
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) tmem_alloc(tmem_holder, TCOLS);
    if (tid == 0) {
        bar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_holder;

    const int i = it.t0 + tid;                         // this thread's target row (preorder index)
    const bool row_ok = i < te;
    const int Di = row_ok ? dist[i] : 0;
    bool ok = true;
    int chunk = 0;
    for (int s0 = tb; s0 < te; s0 += kTileK, ++chunk) {
        // --- A: f(D) tile, row = this thread's target, 64 sources, split hi / lo
#pragma unroll 1
        for (int kg = 0; kg < kTileK / 8; ++kg) {
            __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int j = s0 + kg * 8 + e;
                float f = 0.f;
                if (row_ok && j < te) {
                    int dd = 0;
                    if (j != i) {
                        const int a = min(i, j) + 1, b = max(i, j);
                        const int lv = 31 - __clz(b - a + 1);
                        const int m = min(__ldg(st + int64_t(lv) * n_pre + a), __ldg(st + int64_t(lv) * n_pre + b - (1 << lv) + 1));
                        dd = Di + __ldg(dist + j) - 2 * m;
                    }
                    f = __ldg(ftab + dd);
                }
                split_bf16(f, h[e], l[e]);
            }
            *reinterpret_cast<uint4 *>(Ahi + kmajor_off(tid, kg * 8)) = *reinterpret_cast<const uint4 *>(h);
            *reinterpret_cast<uint4 *>(Alo + kmajor_off(tid, kg * 8)) = *reinterpret_cast<const uint4 *>(l);
        }
        // --- B: field rows of the 64 sources, channels c0 .. c0+NC (hi rows, then lo rows for F32)
        for (int seg = tid; seg < NC * (kTileK / 8); seg += 128) {
            const int n = seg % NC, kg = seg / NC;
            const int c = it.c0 + n;
            __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int j = s0 + kg * 8 + e;
                const float x = (j < te && c < d) ? load_f<T>(F + int64_t(vtx[j]) * d + c) : 0.f;
                split_bf16(x, h[e], l[e]);
            }
            *reinterpret_cast<uint4 *>(B + kmajor_off(n, kg * 8)) = *reinterpret_cast<const uint4 *>(h);
            if (F32) *reinterpret_cast<uint4 *>(B + kmajor_off(NC + n, kg * 8)) = *reinterpret_cast<const uint4 *>(l);
        }
        fence_async_smem();
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
        if (tid == 0) {
#pragma unroll
            for (int ks = 0; ks < kTileK / 16; ++ks) {
                const uint32_t acc = (chunk > 0 || ks > 0) ? 1u : 0u;
                const uint64_t ah = sdesc(smem_addr(Ahi) + ks * 256, 128, 1024);
                const uint64_t al = sdesc(smem_addr(Alo) + ks * 256, 128, 1024);
                const uint64_t bd = sdesc(smem_addr(B) + ks * 256, 128, 1024);
                mma_bf16(tmem, ah, bd, idesc_bf16(kTileM, N1), acc);
                mma_bf16(tmem + N1, al, bd, idesc_bf16(kTileM, N2), acc);
            }
            mma_commit(bar);
        }
        // operands are reused by the next chunk: wait for the MMAs to finish
        const bool done = bar_wait(bar, uint32_t(chunk & 1));
        ok = __syncthreads_and(done ? 1 : 0) != 0;   // CTA-uniform
        fence_after_sync();
        if (!ok) break;
    }
    if (!ok && tid == 0) atomicExch(err, 1);
    // --- epilogue: warp w reads TMEM lanes 32w .. 32w+31 (its 32 targets)
    if (ok && chunk > 0) {
        const uint32_t lane_base = uint32_t(warp * 32) << 16;
#pragma unroll 1
        for (int c = 0; c < NC; c += 16) {
            float a[16], b2[16], c2[16];
            tmem_ld16(tmem + lane_base + c, a);
            if (F32) tmem_ld16(tmem + lane_base + NC + c, b2);
            tmem_ld16(tmem + lane_base + N1 + c, c2);
            if (row_ok) {
                T *dst = out + int64_t(vtx[i]) * d + it.c0 + c;
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    if (it.c0 + c + q < d) {
                        const float v = a[q] + (F32 ? b2[q] : 0.f) + c2[q];
                        if (F32) reinterpret_cast<float *>(dst)[q] = v;
                        else reinterpret_cast<__nv_bfloat16 *>(dst)[q] = __float2bfloat16_rn(v);
                    }
                }
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TCOLS);
}

// Sparse-table level l from level l-1 over the concatenated tree preorders;
// queries never cross a tree boundary, so levels may mix trees.
__global__ void sparse_level(const int32_t *__restrict__ prev, int32_t *__restrict__ next, int64_t n, int half) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        next[i] = (i + half < n) ? min(prev[i], prev[i + half]) : prev[i];
}

// Dynamic shared memory per CTA. It is also what bounds co-resident CTAs, and
// with them the tensor memory in use: 64 columns per CTA for FP32 fields, 128
// for BF16 fields, so BF16 CTAs ask for 48 KB (at most 4 per SM, 512 columns).
template <typename T, int NC>
constexpr size_t dense_smem_bytes() {
    return sizeof(T) == 4 ? 32768 + size_t(2 * NC) * 128 + 16 : 48 * 1024;
}

}  // namespace tc
}  // namespace tfi
