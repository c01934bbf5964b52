// Host-side decomposition planner for StAd-TFI.
//
// Builds the recursion of Algorithm 5 ("Solve") iteratively: for each call S
// with more than s0 vertices it selects a backbone (Algorithm 6,
// "ChooseBackbone", Eq. "stad-score"), decomposes S into the backbone and
// off-backbone components (Algorithm 1), and records per vertex its depth
// d(u) and the grid coordinate of its projection pi(u) (Eq. "projection",
// Eq. "stad-depth"). Calls with at most s0 vertices become dense leaves.
// Everything is on the quantised metric: integer edge lengths q_e >= 1 and
// grid units for depths, coordinates and table sizes.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace tfi {

struct KernelFn {
    int kind = 1;
    std::vector<double> params;
    std::vector<double> table;
    // f(k * delta) in FP64; for a sampled table, NaN beyond its end.
    double grid(int64_t k, double delta) const;
};

struct Call {
    int32_t level, minv, size, kind;   // kind 0 = diameter path, 1 = centroid
    int64_t bb_begin, bb_end;          // backbone p_1..p_m in HostPlan::bb
    int64_t H, L;                      // max depth, backbone length X_m (grid units)
    int64_t rec_begin, rec_end;        // records: backbone first, then components
    int32_t comp_begin, comp_end;      // components in HostPlan::comps
};

struct Comp {
    int32_t call, minv, size;
    int32_t anchor_idx;                // index of the anchor on the backbone
    int64_t H;                         // H_alpha (grid units)
};

struct Rec {
    int32_t v;      // vertex
    int32_t r;      // depth d(v), grid units
    int32_t x;      // coordinate X(pi(v)) on the backbone, grid units
    int32_t comp;   // global component index, -1 on the backbone
};

struct Leaf {
    int32_t level, minv;
    int64_t begin, end;                // range in leaf_vtx (preorder from minv)
    int64_t diam;                      // largest grid distance inside the leaf
};

// One evaluation job: val[i] = sum_j f(r_i + r_j + |x_i - x_j|) * sum[j] over the
// job's keys (a call's cross table G at its occupied bins, Eq. "sumofFFTterms",
// or a component's correction E_alpha, Eq. "stad-E").
struct Job {
    int64_t kb, ke;       // key range
    int32_t maxr, maxx;   // largest depth / coordinate among the keys
    int32_t lp1, lp2;     // log2 FFT sizes (depth, backbone)
    int32_t mode;         // 0 = FFT, 1 = direct, 2 = exponential sweep (inside the call's sweep job),
                          // 3 = Hankel-matrix product on tensor cores, 4 = four-step FFT through
                          // global memory (tables beyond one CTA's shared memory)
    int32_t is_comp;      // 1 for a correction job
};

// Algorithm 7 job: one call. Its A-bins in sw_keys[sb, se) are grouped into m
// runs (one per backbone vertex, ascending coordinate; within a run ascending
// depth) with boundaries sw_run[rb .. rb+m]; its components' b-bins are the
// jobs [cjb, cje).
struct SweepJob {
    int32_t sb, se, rb, m, cjb, cje;
};

struct HostPlan {
    // input
    int32_t n = 0;
    int32_t flags = 0;
    double delta = 1.0;
    KernelFn f;
    int32_t policy = 0, leaf_max = 1, max_channels = 1;
    std::vector<int64_t> ptr;
    std::vector<int32_t> adj;
    std::vector<int64_t> qlen;
    // decomposition
    std::vector<Call> calls;
    std::vector<int32_t> bb;
    std::vector<Rec> recs;
    std::vector<Comp> comps;
    std::vector<Leaf> leaves;
    std::vector<int32_t> leaf_vtx, leaf_dist, leaf_pdist;
    int32_t n_levels = 0;
    // flattened for the device
    std::vector<int32_t> key_r, key_x, key_ptr, key_vtx;   // keys (A-bins, then each component's b-bins, per call)
    std::vector<Job> jobs;
    std::vector<int32_t> vrec_ptr, vrec_akey, vrec_bkey;   // per vertex, its (A-key, b-key) per non-leaf call
    std::vector<int32_t> lgrp_ptr;                         // leaf groups: ranges of leaf_vtx
    std::vector<int32_t> leaf_lo, leaf_hi;                 // per leaf vertex: its leaf's range (absolute)
    std::vector<uint8_t> in_leaf;                          // per vertex: 1 if it lies in a leaf call (backbone
                                                           // vertices of non-leaf calls are complete there)
    // device distance pass (rooted forest + per-record anchor and backbone start)
    std::vector<int32_t> k1_parent, k1_qpar;               // parent (self at a root) and edge length to it
    int32_t k1_maxhop = 0;                                 // largest hop depth below a root
    std::vector<int32_t> rec_anchor, rec_p1;               // per record: pi(v) and the call's p_1
    // exponential-sum sweeps (TFI_PLAN_SWEEP)
    std::vector<int32_t> sw_keys, sw_run;
    std::vector<SweepJob> sweeps;
    std::vector<float> sw_beta, sw_coef;                   // per term: decay per grid unit, coefficient
    int64_t ftab_len = 0;
    int64_t leaf_ftab_len = 1;                             // samples a dense leaf reads: its largest diameter + 1
    int64_t hist_len = 0;                                  // 1 + largest grid distance any pair of a call can have
    // support truncation: every FP32 sample f(k delta) with trunc <= k < trunc_check is zero, so bins at
    // depth >= trunc neither contribute nor receive anything; their table values are zeroed (zero_ranges:
    // [begin, end) key ranges) and the jobs end before them. trunc = -1: no truncation. jobs_full keeps
    // the untruncated jobs (the kernel gradient counts pairs at every distance).
    int64_t trunc = -1, trunc_check = 0;
    std::vector<int32_t> zero_ranges;
    std::vector<Job> jobs_full;
    std::vector<float> ftab;
    // FFT spectra per (lp1, lp2) class, bit-reversed order, scaled by 1/(P1 P2), interleaved re/im
    std::vector<int64_t> spec_class_off;                   // [lp1 * 32 + lp2] -> offset in floats (complex = 2)
    std::vector<float> spectra;
    std::vector<float> twiddle;                            // [h + o] = exp(-2 pi i o / (8 h)), h = 2^L < 2^kTwLog
    double plan_seconds = 0;
};

constexpr int kTwLog = 14;            // largest in-shared-memory FFT: 2^14 complex points
constexpr int kFftMaxLog = 14;
constexpr int kBigMaxLog = 25;        // largest four-step FFT table: 2^25 points
constexpr int kBigMaxInnerLog = 13;   // its backbone axis stays within one block
constexpr int kSpecClasses = 32 * 32; // spectrum classes, indexed lp1 * 32 + lp2

// Split of a four-step FFT table of 2^lp1 x 2^lp2 points (depth outer, backbone
// inner, lp1 >= 1, lp2 <= 13, lp1 + lp2 <= 25): columns of 2^lnA points (pass A / C)
// and blocks of 2^(lp1b + lp2) contiguous points (pass B), lnA + lp1b = lp1. The
// two are balanced (about half the bits each) within columns of at most 2^12 and
// blocks of at most 2^13 points.
struct BigSplit {
    int lnA, lp1b;
};
inline BigSplit big_split(int lp1, int lp2) {
    const int lg = lp1 + lp2;
    int lnA = lg / 2;
    if (lnA < lg - 13) lnA = lg - 13;
    if (lnA > 12) lnA = 12;
    if (lnA > lp1) lnA = lp1;
    return BigSplit{lnA, lp1 - lnA};
}
constexpr int kLeafMax = 1024;        // largest dense leaf (shared-memory sparse table)
constexpr int kLeafGroup = 256;       // small leaves are packed into groups of <= this many vertices
constexpr int64_t kGridMax = int64_t(1) << 30;

// Recompute the f-dependent parts of a built plan (samples, spectra, sweep
// terms) from hp.f. Returns 0 or a TFI_ERR_* code with a message.
int sample_kernel(HostPlan &hp, std::string &err);

// Returns 0 or a TFI_ERR_* code with a message.
int build_plan(HostPlan &hp, int32_t n, int32_t m, const int32_t *u, const int32_t *v, const double *w,
               std::string &err);

}  // namespace tfi
