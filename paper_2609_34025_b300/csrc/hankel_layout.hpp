// Shared-memory layout of one Hankel-evaluator CTA (hankel_tc.cuh). The
// planner uses it to decide which tables qualify, the launch to size dynamic
// shared memory, the kernel to carve it up.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define TFI_HD __host__ __device__
#else
#define TFI_HD
#endif

namespace tfi {

constexpr int kHankelMaxDepths = 64;              // H + 1 <= 64 (MMA K)
constexpr int kHankelMaxRows = 128;               // H + L + 1 <= 128 (MMA N: rows l = q + |s - t|)
constexpr uint32_t kHankelMaxSmem = 227u * 1024u; // one CTA's dynamic shared memory

struct HankelLayout {
    int S;       // rows l = 0 .. H + L
    int NP;      // MMA N: S rounded up to 16
    int KT;      // depths r = 0 .. H rounded up to 8 (MMA K steps of 8)
    int W;       // backbone columns t = 0 .. L
    uint32_t sbo;                                        // bytes between 8-row core-matrix groups
    uint32_t a_bytes, f_bytes;                           // one TF32 operand tile (hi or lo)
    uint32_t f_off, map_off, col_off, acc_off, bar_off, bytes;
};

TFI_HD inline HankelLayout hankel_layout(int H, int L) {
    HankelLayout o;
    o.S = H + L + 1;
    o.NP = (o.S + 15) & ~15;
    o.KT = (H + 8) & ~7;
    o.W = L + 1;
    o.sbo = uint32_t(o.KT) * 32u;                        // KT / 4 core matrices of 128 B per 8 rows
    o.a_bytes = 16u * o.sbo;                             // 128 channel rows
    o.f_bytes = uint32_t(o.NP / 8) * o.sbo;              // NP rows
    o.f_off = 2u * o.a_bytes;                            // Ahi, Alo, then Fhi, Flo
    o.map_off = o.f_off + 2u * o.f_bytes;
    o.col_off = o.map_off + uint32_t(4 * (H + 1) * o.W); // map[r * W + t] -> key or -1
    o.acc_off = (o.col_off + uint32_t(4 * o.W) + 15u) & ~15u;   // col[t]: column t occupied
    const uint32_t acc = L > 0 ? uint32_t(2 * o.S * 128 * 4) : 0u; // accL, accD: S x 128 FP32 each
    o.bar_off = (o.acc_off + acc + 15u) & ~15u;
    o.bytes = o.bar_off + 16u;
    return o;
}

TFI_HD inline bool hankel_fits(int H, int L) {
    return H + 1 <= kHankelMaxDepths && H + L + 1 <= kHankelMaxRows && hankel_layout(H, L).bytes <= kHankelMaxSmem;
}

TFI_HD inline uint32_t hankel_tmem_cols(int np) { return np <= 32 ? 32u : np <= 64 ? 64u : 128u; }

}  // namespace tfi
