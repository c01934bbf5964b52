// C ABI of libtfi (include/tfi.h): plan upload, apply orchestration, export.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>
#include <queue>
#include <cstdint>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "dense_tc.cuh"
#include "grad.cuh"
#include "hankel_tc.cuh"
#include "leaf_tc.cuh"
#include "leaf_tc32.cuh"
#include "table_tc32.cuh"
#include "kernels.cuh"
#include "fft_x2.cuh"
#include "fft_big.cuh"
#include "planner.hpp"
#include "tfi.h"

namespace {

thread_local std::string g_err;

tfi_status fail(tfi_status code, const std::string &msg) {
    g_err = msg;
    return code;
}

#define TFI_CUDA(call)                                                                         \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(TFI_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));     \
    } while (0)

struct WorkLists {
    // FFT items grouped by log2(P1 P2): one launch per class
    std::vector<int> fft_lnp;
    std::vector<int> fft_count;
    std::vector<int> fft_npair;
    std::vector<int64_t> fft_off;
    tfi::dev::FftItem *d_fft = nullptr;
    tfi::dev::DirItem *d_dir = nullptr;
    int n_dir = 0;
    // direct jobs on the tensor cores: (kb, ke, two-dimensional, 0), grouped by CTA (each
    // CTA's largest first)
    int4 *d_tab = nullptr;
    int32_t *d_tab_ptr = nullptr;  // CTA b takes d_tab[d_tab_ptr[b] .. d_tab_ptr[b + 1])
    int n_tab = 0, tab_grid = 0, tab_max_keys = 1, tab_fts = 1;
    // Hankel-matrix jobs: one item per (job, 128-channel block), one launch
    tfi::tc::HankelItem *d_hk = nullptr;
    int n_hk = 0;
    size_t hk_smem = 0;
    // four-step FFT tables: one item per (table, channel pair); batches that fit the plan's
    // buffer, each a run of size-class segments [i0, i1) of d_big
    struct BigSeg {
        tfi::dev::BigGeom g;
        int64_t i0, i1, max_nk;
    };
    tfi::dev::BigItem *d_big = nullptr;
    std::vector<std::vector<BigSeg>> big_batches;
    int64_t big_elems = 0;  // buffer elements (16 bytes: two channel pairs) the largest batch needs
};

constexpr int64_t kBigBatchBytes = int64_t(4) << 30;  // four-step FFT buffer of a plan, at most
constexpr int kLeafTc32MinChannels = 16;       // FP32 fields: tensor-core big leaves from this d,
constexpr double kLeafTc32MinShare = 0.25;     // when the leaves are at least this share of the leaf
                                               // and table flops: its persistent CTAs hold most of
                                               // an SM's registers, which the concurrent table
                                               // stages then miss (N = 2^20 caterpillar, leaves 3 %
                                               // of the flops: 63.5 against 57.1 ms per step; random
                                               // tree, 34 %: 3.03 against 3.07-3.13 ms)
constexpr int kTable32MinChannels = 17;        // direct tables on the tensor cores from this d: one
                                               // f operand for all channels where the ALU kernel
                                               // needs two or more 16-channel passes (N = 2^20:
                                               // 0.66 against 0.96 ms at d = 64, 0.25 against
                                               // 0.24 ms at d = 16 on the random tree's tables)
constexpr int kTable32BigKeys = 512;           // and at d = 16 for tables of this many bins or more
                                               // (the 2^20 caterpillar: 52.1 against 57.1 ms)
constexpr size_t kLeaf32SmemMax = 110 * 1024;  // tensor-core leaf / table CTAs: two per SM (with the
                                               // static and reserved bytes)

}  // namespace

struct tfi_plan_s {
    tfi::HostPlan hp;
    bool on_device = false;
    int device = -1;
    int64_t dev_bytes = 0;
    std::vector<void *> allocs;
    // device arrays
    int32_t *key_r = nullptr, *key_x = nullptr, *key_ptr = nullptr, *key_vtx = nullptr;
    tfi::dev::JobDev *jobs = nullptr;
    // per gather position i (vertex gorder[i]): its (A-key, b-key) pairs, one per non-leaf call
    int32_t *vrec_ptr = nullptr, *vrec_akey = nullptr, *vrec_bkey = nullptr;
    int32_t *lgrp_ptr = nullptr, *leaf_vtx = nullptr, *leaf_dist = nullptr, *leaf_pdist = nullptr;
    int32_t *leaf_lo = nullptr, *leaf_hi = nullptr;
    uint8_t *in_leaf = nullptr;   // per gather position: the vertex has a leaf term
    int32_t *leaf_row = nullptr;  // per leaf slot: the lbuf row of its vertex (its gather position)
    int32_t *gorder = nullptr;  // vertices in depth-first preorder of the forest (gather order)
    int32_t max_gs = 0, n_groups = 0;
    // FP32-ALU leaves: groups of consecutive small leaves (one thread per target) and big leaves of
    // at least kLeafWarpMin vertices (one warp per 32 targets, broadcast source loads)
    int32_t *sgrp_ptr = nullptr, *big_lo = nullptr, *big_hi = nullptr;  // sgrp_ptr: [begin, end) per group
    int32_t n_sgroups = 0, max_sgs = 1, n_big = 0, max_big = 1;
    // big leaves packed into CTAs of leaf_warp_kernel: CTA b runs leaves big_lo/hi[big_ptr[b] ..
    // big_ptr[b + 1]), at most 8 warps of 64 targets and max_big vertices in all
    int32_t *big_ptr = nullptr;
    float *ftab = nullptr;
    float2 *spectra = nullptr, *twiddle = nullptr;
    float4 *twiddle_b = nullptr;  // the twiddles, each value as (re, re, im, im)
    float *kbuf = nullptr, *vbuf = nullptr, *lbuf = nullptr;
    // four-step FFT tables: the buffer of one batch (grown on demand by build_work) and the two
    // twiddle tables exp(-2 pi i j / 2^13), exp(-2 pi i j / 2^26), j < 2^13
    ulonglong2 *big_buf = nullptr;  // 16-byte elements: one point of two channel pairs
    float2 *big_tw_hi = nullptr, *big_tw_lo = nullptr;
    int64_t big_cap = 0;
    int32_t n_big_jobs = 0;
    // bin sums by segments of at most kBucketSeg members (see bucket_seg_kernel)
    int32_t *seg_ptr = nullptr, *seg_dst = nullptr, *mb_key = nullptr, *mb_ptr = nullptr;
    int64_t n_segs = 0, n_multi = 0;
    float *sbuf = nullptr;
    float *sk_buf = nullptr;  // Sinkhorn: K x (n x max_channels), allocated on first use
    // kernel gradient (built on first use)
    bool grad_ready = false;
    int32_t n_gjobs = 0, n_gleaves = 0, n_gseg = 0, g_max_lnp = 0, g_nblk = 1;
    int32_t g_leaf_max_n = 1, g_leaf_max_hl = 1;   // largest leaf and leaf histogram (one-pass leaf kernel)
    bool g_leaf_onepass = false;                    // its shared memory fits: no per-pair buffers
    int32_t *g_leaf_S = nullptr;                    // per leaf: the fixed-point scale exponent
    unsigned long long *g_h64 = nullptr;            // the leaves' fixed-point histograms (channel-block CTAs)
    int64_t g_leaf_hbase = 0, g_leaf_hlen = 0;      // their range in g_hist
    int64_t *g_ditems = nullptr;
    int32_t *g_djobs = nullptr, n_gditems = 0, n_gdjobs = 0;
    int32_t g_dir_max_k = 1, g_dir_max_nk = 1;   // direct gradient jobs: largest histogram and key count
    int32_t *g_fft1d = nullptr;                    // one-dimensional FFT gradient jobs (paired-FP32 kernel),
    int32_t n_gfft1d = 0;                          // grouped by transform size: class ln holds
    std::vector<int32_t> g_fft1d_cls;              // g_fft1d[cls[ln] .. cls[ln + 1]) (ln = 0 .. 14)
    float *g_M = nullptr;
    tfi::grad::GradJob *g_jobs = nullptr;
    int32_t *g_leaf_ptr = nullptr, *g_hist_len = nullptr, *g_seg_len = nullptr, *g_pdst = nullptr;
    int64_t *g_pair_off = nullptr, *g_hist_off = nullptr, *g_seg_off = nullptr;
    float *g_seg_sign = nullptr, *g_hist = nullptr, *g_pval = nullptr, *g_gbuf = nullptr;
    double *g_C = nullptr, *g_params = nullptr, *g_dtheta = nullptr;
    // exponential sweeps
    tfi::dev::SweepJobDev *sw_jobs = nullptr;
    int32_t *sw_keys = nullptr, *sw_run = nullptr, *sw_ejobs = nullptr;
    float *sw_beta = nullptr, *sw_coef = nullptr, *sw_scratch = nullptr;
    int32_t n_sweeps = 0, n_sw_ejobs = 0, sw_terms = 0;
    void *stage_in = nullptr, *stage_out = nullptr;
    // tfi_apply_host_many: two staging slots (in, out), copy-in and copy-out streams, and per slot
    // the events that order copy-in -> apply -> copy-out and the reuse of a slot two fields later
    void *pipe_in[2] = {nullptr, nullptr}, *pipe_out[2] = {nullptr, nullptr};
    cudaStream_t pipe_cin = nullptr, pipe_cout = nullptr;
    cudaEvent_t ev_in_ready[2] = {nullptr, nullptr}, ev_in_free[2] = {nullptr, nullptr};
    cudaEvent_t ev_out_ready[2] = {nullptr, nullptr}, ev_out_free[2] = {nullptr, nullptr};
    int32_t *dev_rec_r = nullptr, *dev_rec_x = nullptr;  // record keys computed on the device at plan time
    // dense tensor-core evaluation (built on first use): per-tree preorder, root
    // distances, sparse table of parent distances, f samples up to the largest diameter
    bool dense_ready = false;
    int32_t dense_trees = 0, dense_levels = 0, dense_max_tree = 0;
    int32_t *dn_tree_ptr = nullptr, *dn_vtx = nullptr, *dn_dist = nullptr, *dn_st = nullptr, *dn_err = nullptr;
    float *dn_ftab = nullptr;
    int64_t dense_ftab_len = 0;
    std::vector<int32_t> dn_tree_ptr_h;
    double device_keys_ms = 0.0;
    int32_t n_hankel = 0;           // jobs evaluated by the Hankel-matrix product
    int32_t *hk_err = nullptr;      // [0]: a Hankel CTA, [1]: a tensor-core leaf CTA whose bounded MMA wait gave up,
                                    // [2]: the last tfi_selftest_wait gave up
    tfi::tc::LeafTile *leaf_tiles = nullptr;  // 128-row tiles of the leaf groups (tensor-core leaves)
    int32_t n_leaf_tiles = 0;
    int2 *leaf32 = nullptr;                 // leaves of >= kLeafWarpMin vertices as [lo, hi), grouped by CTA
    int32_t n_leaf32 = 0, max_leaf32 = 1;   // (the FP32 tensor-core leaf kernel)
    int32_t *leaf32_ptr = nullptr;          // CTA b takes leaf32[leaf32_ptr[b] .. leaf32_ptr[b + 1])
    int32_t leaf32_grid = 0;
    double leaf_share = 0;                  // dense-leaf flops / all leaf and table flops (per channel)
    std::map<int, WorkLists> work;  // per channel count d
    int32_t fft_cta_points = 1 << 13;  // tfi_options.fft_cta_points (0 there: this default)
    // tfi_apply_static: its work lists without per-call host copies. Direct items do not depend
    // on d; FFT jobs are kept by size class and expanded into (job, pair block) items on the
    // device at each call, into the static workspace
    tfi::dev::DirItem *st_dir = nullptr;
    int32_t n_st_dir = 0;
    int32_t *st_fft_job = nullptr;
    // support truncation: key ranges whose table values are zero
    int32_t *zero_ranges = nullptr;
    int32_t n_zero_ranges = 0;
    std::vector<int> st_cls_lnp;
    std::vector<int32_t> st_cls_joff, st_cls_njobs;
    // fork/join inside an apply: leaf terms and direct jobs run on their own
    // streams, concurrently with the bin sums and FFT jobs
    // aux[0]: leaves, aux[1]: direct / Hankel jobs, aux[2]: the critical path bin sums -> FFT jobs
    cudaStream_t aux[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t ev_crit = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_leaf = nullptr, ev_bucket = nullptr, ev_dir = nullptr;
    // stage profiling (CUDA events on the apply stream)
    bool profiling = false;
    bool serialize = false;  // profiling mode 2: every stage on the caller's stream
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    struct StageRec {
        int stage;
        int launches;
        cudaEvent_t a, b;
    };
    std::vector<StageRec> prof;
    cudaEvent_t next_event() {
        if (ev_used == ev_pool.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            ev_pool.push_back(e);
        }
        return ev_pool[ev_used++];
    }

    template <typename T>
    tfi_status upload(T **dst, const std::vector<T> &src) {
        if (src.empty()) {
            *dst = nullptr;
            return TFI_OK;
        }
        void *p = nullptr;
        if (cudaMalloc(&p, src.size() * sizeof(T)) != cudaSuccess)
            return fail(TFI_ERR_OOM, "cudaMalloc failed while uploading the plan");
        allocs.push_back(p);
        dev_bytes += int64_t(src.size() * sizeof(T));
        TFI_CUDA(cudaMemcpy(p, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
        *dst = static_cast<T *>(p);
        return TFI_OK;
    }
    tfi_status alloc(void **dst, size_t bytes) {
        if (bytes == 0) bytes = 16;
        if (cudaMalloc(dst, bytes) != cudaSuccess) return fail(TFI_ERR_OOM, "cudaMalloc failed for the workspace");
        allocs.push_back(*dst);
        dev_bytes += int64_t(bytes);
        return TFI_OK;
    }
    ~tfi_plan_s() {
        for (cudaEvent_t e : {ev_fork, ev_leaf, ev_bucket, ev_dir, ev_crit, ev_in_ready[0], ev_in_ready[1],
                              ev_in_free[0], ev_in_free[1], ev_out_ready[0], ev_out_ready[1], ev_out_free[0],
                              ev_out_free[1]})
            if (e) cudaEventDestroy(e);
        for (cudaStream_t st : {pipe_cin, pipe_cout})
            if (st) cudaStreamDestroy(st);
        for (cudaStream_t st : aux)
            if (st) cudaStreamDestroy(st);
        for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
        for (auto &kv : work) {
            cudaFree(kv.second.d_fft);
            cudaFree(kv.second.d_dir);
            cudaFree(kv.second.d_tab);
            cudaFree(kv.second.d_tab_ptr);
            cudaFree(kv.second.d_hk);
            cudaFree(kv.second.d_big);
        }
        cudaFree(big_buf);
        for (void *p : allocs) cudaFree(p);
    }
};

namespace {

constexpr int kFftThreads = 256;
constexpr int kFftSmemPairPoints = 1 << 13;  // default points x pairs per CTA (64 KB) for classes below 2^13

// Channel pairs per CTA of the shared-memory FFT for a class of 2^lnp points: up to
// cta_points / 2^lnp (tfi_options.fft_cta_points; one pair from 2^13 points on).
int fft_pairs_per_cta(int lnp, int pairs, int cta_points) {
    const int cap = lnp >= 13 ? 1 : std::max(1, cta_points >> lnp);
    return std::max(1, std::min(pairs, cap));
}

int device_sms();

// Work of one leaf or direct job in the persistent tensor-core kernels: its 128-row tiles x
// 32-source chunks, plus a few chunks' worth of per-item staging.
double tc32_cost(int n) { return std::ceil(n / 128.0) * std::ceil(n / 32.0) + 4.0; }

// Longest-processing-time-first assignment of items (sorted largest first) to `ctas` persistent
// CTAs: each item goes to the CTA with the least work so far (the lowest index among equals).
// `grouped` receives the items CTA by CTA (each CTA's in the original, descending order) and
// `ptr` the ctas + 1 offsets into it. Within a few percent of the optimum where round-robin
// over the sorted list leaves the first CTAs 10-20 % above the mean.
template <typename Item, typename Size>
void lpt_schedule(const std::vector<Item> &items, int ctas, Size size, std::vector<Item> &grouped,
                  std::vector<int32_t> &ptr) {
    std::vector<std::vector<int32_t>> per(size_t(std::max(ctas, 0)));
    using Load = std::pair<double, int>;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int b = 0; b < ctas; ++b) heap.push({0.0, b});
    for (size_t i = 0; i < items.size() && ctas > 0; ++i) {
        const Load l = heap.top();
        heap.pop();
        per[size_t(l.second)].push_back(int32_t(i));
        heap.push({l.first + tc32_cost(size(items[i])), l.second});
    }
    grouped.clear();
    ptr.assign(1, 0);
    for (int b = 0; b < ctas; ++b) {
        for (int32_t i : per[size_t(b)]) grouped.push_back(items[size_t(i)]);
        ptr.push_back(int32_t(grouped.size()));
    }
}

tfi_status build_work(tfi_plan_t p, int d, WorkLists **out) {
    auto it = p->work.find(d);
    if (it != p->work.end()) {
        *out = &it->second;
        return TFI_OK;
    }
    WorkLists wl;
    const int pairs = (d + 1) / 2;
    std::map<int, std::vector<tfi::dev::FftItem>> by_class;
    std::vector<tfi::dev::DirItem> dir;
    std::vector<int4> tab;
    std::vector<tfi::tc::HankelItem> hk;
    uint32_t hk_cols = 32;
    const auto &jobs = p->hp.jobs;
    const bool tab_alu = (p->hp.flags & TFI_PLAN_TABLES_ALU) != 0;
    for (size_t j = 0; j < jobs.size(); ++j) {
        const tfi::Job &jb = jobs[j];
        if (jb.ke == jb.kb || jb.mode == 2 || jb.mode == 4) continue;
        if (jb.mode == 3) {
            const tfi::HankelLayout lay = tfi::hankel_layout(jb.maxr, jb.maxx);
            wl.hk_smem = std::max(wl.hk_smem, size_t(lay.bytes));
            hk_cols = std::max(hk_cols, tfi::hankel_tmem_cols(lay.NP));
            for (int c0 = 0; c0 < d; c0 += 128)
                hk.push_back(tfi::tc::HankelItem{int32_t(jb.kb), int32_t(jb.ke), c0, jb.maxr, jb.maxx, {0, 0, 0}});
        } else if (jb.mode == 0) {
            const int lnp = jb.lp1 + jb.lp2;
            const int np = fft_pairs_per_cta(lnp, pairs, p->fft_cta_points);
            for (int p0 = 0; p0 < pairs; p0 += np)
                by_class[lnp].push_back(tfi::dev::FftItem{int32_t(j), p0, std::min(np, pairs - p0)});
        } else if (!tab_alu && jb.ke - jb.kb >= tfi::tc::kTab32MinKeys && jb.ke - jb.kb <= tfi::tc::kTab32MaxKeys &&
                   (d >= kTable32MinChannels || (d == 16 && jb.ke - jb.kb >= kTable32BigKeys))) {
            tab.push_back(make_int4(int32_t(jb.kb), int32_t(jb.ke), jb.maxx > 0 ? 1 : 0, 0));
            wl.tab_max_keys = std::max(wl.tab_max_keys, int(jb.ke - jb.kb));
            wl.tab_fts = std::max(wl.tab_fts, 2 * jb.maxr + jb.maxx + 1);
        } else {
            for (int64_t q = jb.kb; q < jb.ke; q += 64) dir.push_back(tfi::dev::DirItem{int32_t(j), int32_t(q)});
        }
    }
    std::stable_sort(tab.begin(), tab.end(), [](int4 a, int4 b) { return a.y - a.x > b.y - b.x; });
    wl.n_tab = int(tab.size());
    if (!tab.empty()) {
        // persistent: two CTAs per SM (their tensor memory), jobs assigned longest first
        wl.tab_grid = std::min(wl.n_tab, 2 * device_sms());
        std::vector<int4> grouped;
        std::vector<int32_t> ptr;
        lpt_schedule(tab, wl.tab_grid, [](int4 a) { return a.y - a.x; }, grouped, ptr);
        TFI_CUDA(cudaMalloc(&wl.d_tab, grouped.size() * sizeof(grouped[0])));
        TFI_CUDA(cudaMemcpy(wl.d_tab, grouped.data(), grouped.size() * sizeof(grouped[0]), cudaMemcpyHostToDevice));
        TFI_CUDA(cudaMalloc(&wl.d_tab_ptr, ptr.size() * sizeof(ptr[0])));
        TFI_CUDA(cudaMemcpy(wl.d_tab_ptr, ptr.data(), ptr.size() * sizeof(ptr[0]), cudaMemcpyHostToDevice));
    }
    std::vector<tfi::dev::FftItem> all;
    for (auto &kv : by_class) {
        wl.fft_lnp.push_back(kv.first);
        wl.fft_count.push_back(int(kv.second.size()));
        wl.fft_npair.push_back(fft_pairs_per_cta(kv.first, pairs, p->fft_cta_points));
        wl.fft_off.push_back(int64_t(all.size()));
        all.insert(all.end(), kv.second.begin(), kv.second.end());
    }
    if (!all.empty()) {
        TFI_CUDA(cudaMalloc(&wl.d_fft, all.size() * sizeof(all[0])));
        TFI_CUDA(cudaMemcpy(wl.d_fft, all.data(), all.size() * sizeof(all[0]), cudaMemcpyHostToDevice));
    }
    wl.n_dir = int(dir.size());
    if (!dir.empty()) {
        TFI_CUDA(cudaMalloc(&wl.d_dir, dir.size() * sizeof(dir[0])));
        TFI_CUDA(cudaMemcpy(wl.d_dir, dir.data(), dir.size() * sizeof(dir[0]), cudaMemcpyHostToDevice));
    }
    wl.n_hk = int(hk.size());
    if (!hk.empty()) {
        // shared memory also caps co-resident CTAs, and with them the tensor memory
        // they allocate: at most 512 / hk_cols CTAs may fit on an SM (228 KB each)
        const size_t max_ctas = 512 / hk_cols;
        wl.hk_smem = std::max(wl.hk_smem, size_t(228 * 1024) / (max_ctas + 1));
        TFI_CUDA(cudaMalloc(&wl.d_hk, hk.size() * sizeof(hk[0])));
        TFI_CUDA(cudaMemcpy(wl.d_hk, hk.data(), hk.size() * sizeof(hk[0]), cudaMemcpyHostToDevice));
    }
    {
        // four-step FFT tables by size class, one item per plane of four channels, in batches whose
        // arrays fit kBigBatchBytes (and 65535 items: the grid rows of the scatter / gather launches)
        std::map<int, std::vector<int32_t>> big_cls;
        for (size_t j = 0; j < jobs.size(); ++j)
            if (jobs[j].mode == 4 && jobs[j].ke > jobs[j].kb) big_cls[jobs[j].lp1 * 32 + jobs[j].lp2].push_back(int32_t(j));
        std::vector<tfi::dev::BigItem> items;
        std::vector<WorkLists::BigSeg> cur;
        int64_t used = 0, first = 0;
        const int64_t cap = kBigBatchBytes / int64_t(sizeof(ulonglong2));
        const int planes = (d + 3) / 4;
        for (auto &kv : big_cls) {
            const int lp1 = kv.first / 32, lp2 = kv.first % 32;
            const tfi::BigSplit sp = tfi::big_split(lp1, lp2);
            const tfi::dev::BigGeom g{lp1, lp2, sp.lnA, sp.lp1b};
            const int64_t P = int64_t(1) << (lp1 + lp2);
            const int64_t spec = p->hp.spec_class_off[size_t(kv.first)] / 2;
            for (int32_t j : kv.second) {
                const tfi::Job &jb = jobs[size_t(j)];
                for (int pr = 0; pr < planes; ++pr) {
                    if (!cur.empty() && (used + P > cap || int64_t(items.size()) - first >= 65535)) {
                        wl.big_batches.push_back(cur);
                        cur.clear();
                        used = 0;
                    }
                    if (cur.empty()) first = int64_t(items.size());
                    if (cur.empty() || cur.back().g.lp1 != lp1 || cur.back().g.lp2 != lp2)
                        cur.push_back(WorkLists::BigSeg{g, int64_t(items.size()), int64_t(items.size()), 0});
                    items.push_back(tfi::dev::BigItem{used, spec, int32_t(jb.kb), int32_t(jb.ke), pr, jb.maxr});
                    used += P;
                    cur.back().i1 = int64_t(items.size());
                    cur.back().max_nk = std::max<int64_t>(cur.back().max_nk, jb.ke - jb.kb);
                    wl.big_elems = std::max(wl.big_elems, used);
                }
            }
        }
        if (!cur.empty()) wl.big_batches.push_back(cur);
        if (!items.empty()) {
            TFI_CUDA(cudaMalloc(&wl.d_big, items.size() * sizeof(items[0])));
            TFI_CUDA(cudaMemcpy(wl.d_big, items.data(), items.size() * sizeof(items[0]), cudaMemcpyHostToDevice));
        }
        if (wl.big_elems > p->big_cap) {
            // grow the plan's buffer (stream-ordered work on the old one has to finish first)
            TFI_CUDA(cudaDeviceSynchronize());
            cudaFree(p->big_buf);
            p->dev_bytes -= p->big_cap * int64_t(sizeof(ulonglong2));
            p->big_buf = nullptr;
            p->big_cap = 0;
            if (cudaMalloc(&p->big_buf, size_t(wl.big_elems) * sizeof(ulonglong2)) != cudaSuccess) {
                cudaFree(wl.d_big);
                return fail(TFI_ERR_OOM, "cudaMalloc failed for the four-step FFT buffer");
            }
            p->big_cap = wl.big_elems;
            p->dev_bytes += p->big_cap * int64_t(sizeof(ulonglong2));
        }
    }
    auto res = p->work.emplace(d, wl);
    *out = &res.first->second;
    return TFI_OK;
}

// (a4, a5) tables beyond shared memory: per batch and size class, zero the rows pass A reads,
// scatter the bin sums, the three passes of the four-step correlation, read the bins back
void launch_big(tfi_plan_t p, const WorkLists &wl, int d, cudaStream_t s) {
    for (const auto &batch : wl.big_batches) {
        for (const WorkLists::BigSeg &sg : batch) {
            const tfi::dev::BigGeom g = sg.g;
            const unsigned n_it = unsigned(sg.i1 - sg.i0);
            const tfi::dev::BigItem *it = wl.d_big + sg.i0;
            const int64_t BLK = int64_t(1) << (g.lp1b + g.lp2), NA = int64_t(1) << g.lnA;
            const int64_t P = BLK * NA;
            const unsigned gz = unsigned(std::min<int64_t>(256, std::max<int64_t>(1, (P / 2 + BLK + 255) / 256)));
            const unsigned gs = unsigned(std::min<int64_t>(64, std::max<int64_t>(1, (sg.max_nk + 255) / 256)));
            tfi::dev::big_zero<<<dim3(gz, n_it), 256, 0, s>>>(it, g, p->big_buf);
            tfi::dev::big_scatter<<<dim3(gs, n_it), 256, 0, s>>>(it, g, p->key_r, p->key_x, d, p->kbuf, p->big_buf);
            const int lcg = tfi::dev::big_lcg(g), lnb = tfi::dev::big_lnb(g);
            const size_t smem_c = (size_t(NA) << lcg) * sizeof(ulonglong2);
            const size_t smem_b = (size_t(BLK) << lnb) * sizeof(ulonglong2);
            const unsigned grid_c = unsigned(n_it * (BLK >> lcg)), grid_b = unsigned(n_it * (NA >> lnb));
            tfi::dev::big_columns<false><<<grid_c, 256, smem_c, s>>>(it, g, lcg, p->big_buf, p->twiddle, p->big_tw_hi,
                                                                    p->big_tw_lo);
            tfi::dev::big_blocks<<<grid_b, 256, smem_b, s>>>(it, int(n_it), g, lnb, p->big_buf, p->spectra, p->twiddle,
                                                             reinterpret_cast<const ulonglong2 *>(p->twiddle_b),
                                                             p->big_tw_hi, p->big_tw_lo);
            tfi::dev::big_columns<true><<<grid_c, 256, smem_c, s>>>(it, g, lcg, p->big_buf, p->twiddle, p->big_tw_hi,
                                                                   p->big_tw_lo);
            tfi::dev::big_gather<<<dim3(gs, n_it), 256, 0, s>>>(it, g, p->key_r, p->key_x, d, p->big_buf, p->vbuf);
        }
    }
}

int big_launches(const WorkLists &wl) {
    int n = 0;
    for (const auto &b : wl.big_batches) n += 6 * int(b.size());
    return n;
}

constexpr int32_t kBucketSeg = 32;  // members per bin-sum segment

constexpr int kMaxDevices = 256;
std::atomic<int> g_sm_count[kMaxDevices] = {};

// Streaming multiprocessors of the current device (read once per device).
int device_sms() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 148;
    int v = g_sm_count[dev].load(std::memory_order_relaxed);
    if (v <= 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
        g_sm_count[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

// Grid of a grid-stride kernel: enough CTAs for the work, at most 32 per SM.
int grid_for(int64_t work, int threads) {
    const int64_t b = (work + threads - 1) / threads;
    return int(std::max<int64_t>(1, std::min<int64_t>(b, int64_t(device_sms()) * 32)));
}

constexpr int kLeafWarpThreads = 256;  // leaf_warp_kernel CTAs: 8 warps

// Packs the big leaves into CTAs of leaf_warp_kernel, largest leaf first: each leaf
// needs ceil(size / 64) warps (64 targets per warp); a CTA takes leaves while their
// warps fit in its 8 and their vertices in max(largest leaf, 512), best fit by free
// warps among the open CTAs. Leaves larger than 512 vertices get a CTA of their own.
void pack_big_leaves(const std::vector<int32_t> &lo, const std::vector<int32_t> &hi, std::vector<int32_t> &bptr,
                     std::vector<int32_t> &blo, std::vector<int32_t> &bhi, int32_t *cap_out) {
    constexpr int kWarps = kLeafWarpThreads / 32, kPer = 32 * tfi::dev::kLeafWarpTargets;
    const size_t nl = lo.size();
    std::vector<size_t> ord(nl);
    std::iota(ord.begin(), ord.end(), size_t(0));
    std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return hi[a] - lo[a] > hi[b] - lo[b]; });
    int32_t cap = kWarps * kPer;
    for (size_t i = 0; i < nl; ++i) cap = std::max(cap, hi[i] - lo[i]);
    struct Bin {
        int warps, verts;
        std::vector<size_t> leaves;
    };
    std::vector<Bin> bins;
    std::vector<std::vector<size_t>> open(kWarps);  // open[r]: bins with r free warps (r >= 1)
    for (size_t i : ord) {
        const int n = hi[i] - lo[i];
        const int w = std::min(kWarps, (n + kPer - 1) / kPer);
        size_t pick = SIZE_MAX;
        for (int r = w; r < kWarps && pick == SIZE_MAX; ++r)
            if (!open[r].empty() && bins[open[r].back()].verts + n <= cap) {
                pick = open[r].back();
                open[r].pop_back();
            }
        if (pick == SIZE_MAX) {
            pick = bins.size();
            bins.push_back(Bin{0, 0, {}});
        }
        Bin &b = bins[pick];
        b.warps += w;
        b.verts += n;
        b.leaves.push_back(i);
        if (n <= kWarps * kPer && b.warps < kWarps) open[kWarps - b.warps].push_back(pick);
    }
    bptr.assign(1, 0);
    blo.clear();
    bhi.clear();
    for (const Bin &b : bins) {
        for (size_t i : b.leaves) {
            blo.push_back(lo[i]);
            bhi.push_back(hi[i]);
        }
        bptr.push_back(int32_t(blo.size()));
    }
    *cap_out = cap;
}

constexpr int kLeafFtabSmemMax = 12288;  // f samples staged in shared memory up to this many

// big = false: only the small leaves (the big ones go to the tensor cores)
// returns the number of kernels launched
template <int CH, typename T>
int launch_leaf(tfi_plan_t p, const T *F, float *lbuf, int d, cudaStream_t s, bool big = true) {
    int launched = 0;
    // leaves look f up at their own pair distances only: stage that prefix of the samples
    const int fts = p->hp.leaf_ftab_len <= kLeafFtabSmemMax ? int(p->hp.leaf_ftab_len) : 0;
    if (big && p->n_big > 0) {
        const size_t smem = tfi::dev::leaf_warp_smem_bytes(p->max_big, CH, fts);
        dim3 grid(p->n_big, (d + CH - 1) / CH);
        auto k = fts > 0 ? tfi::dev::leaf_warp_kernel<T, CH, true> : tfi::dev::leaf_warp_kernel<T, CH, false>;
        k<<<grid, kLeafWarpThreads, smem, s>>>(p->big_ptr, p->big_lo, p->big_hi, p->leaf_vtx, p->leaf_dist,
                                               p->leaf_pdist, F, d, p->ftab, fts, lbuf, p->leaf_row, p->max_big);
        ++launched;
    }
    if (p->n_sgroups > 0) {
        const size_t smem = tfi::dev::leaf_smem_bytes(p->max_sgs, CH, fts);
        dim3 grid(p->n_sgroups, (d + CH - 1) / CH);
        auto k = fts > 0 ? tfi::dev::leaf_kernel<T, CH, true> : tfi::dev::leaf_kernel<T, CH, false>;
        k<<<grid, 256, smem, s>>>(p->sgrp_ptr, p->leaf_vtx, p->leaf_dist, p->leaf_pdist, p->leaf_lo, p->leaf_hi, F, d,
                                  p->ftab, fts, lbuf, p->leaf_row, p->max_sgs);
        ++launched;
    }
    return launched;
}

constexpr int kLeafTcFtabSmem = 4096;  // f samples staged in shared memory by the tensor-core leaf kernel
constexpr int kLeafTcMinChannels = 64;  // below this the FP32-ALU leaf kernel is used

template <typename T, int NB>
size_t leaf_tc_smem(int fts) {
    constexpr uint32_t tcols = NB <= 32 ? 32u : uint32_t(NB);
    const size_t max_ctas = 512 / tcols;  // tensor memory per SM bounds co-resident CTAs
    return std::max(size_t(tfi::tc::leaf_tc_layout(NB, sizeof(T) == 4, fts).bytes), size_t(228 * 1024) / (max_ctas + 1));
}

template <typename T, int NB>
void launch_leaf_tc_nb(tfi_plan_t p, const T *F, float *lbuf, int d, cudaStream_t s) {
    const int fts = p->hp.leaf_ftab_len <= kLeafTcFtabSmem ? int(p->hp.leaf_ftab_len) : 0;
    dim3 grid(unsigned(p->n_leaf_tiles), unsigned((d + NB - 1) / NB));
    tfi::tc::leaf_tc_kernel<T, NB><<<grid, 256, leaf_tc_smem<T, NB>(fts), s>>>(
        p->leaf_tiles, p->leaf_vtx, p->leaf_dist, p->leaf_pdist, p->leaf_lo, p->leaf_hi, F, d, p->ftab, fts, lbuf,
        p->leaf_row, p->hk_err + 1);
}

// Tensor-core leaves for BF16 fields: NB = channels per CTA (TMEM columns), the next power of two
// >= d, from 64 to 256; one chained FP32 accumulator per tile (within the BF16 bound). FP32 fields
// use leaf_tc32_kernel instead: this kernel's accumulation over the ~1000 chained MMAs of a large
// leaf measured 6.5e-4 normwise on a slowly decaying kernel, beyond the FP32 bound of 1e-4.
// Returns the number of kernels launched.
int launch_leaf_tc(tfi_plan_t p, const __nv_bfloat16 *F, float *lbuf, int d, cudaStream_t s) {
    if (p->n_leaf_tiles == 0) return 0;
    using B = __nv_bfloat16;
    if (d > 128) launch_leaf_tc_nb<B, 256>(p, F, lbuf, d, s);
    else if (d > 64) launch_leaf_tc_nb<B, 128>(p, F, lbuf, d, s);
    else launch_leaf_tc_nb<B, 64>(p, F, lbuf, d, s);
    return 1;
}

// FP32 leaves of >= kLeafWarpMin vertices on the tensor cores: NB channels per CTA


template <int NB>
void launch_leaf_tc32_nb(tfi_plan_t p, const float *F, float *lbuf, int d, cudaStream_t s) {
    int fts = int(p->hp.leaf_ftab_len);
    if (tfi::tc::leaf_tc32_layout(NB, p->max_leaf32, fts).bytes > kLeaf32SmemMax) fts = 0;
    // no shared-memory padding: the registers (288 threads x 96) already keep it to two CTAs per SM,
    // which its tensor memory holds, and the rest of the SM stays open to the kernels that run
    // beside it (a four-step FFT CTA takes 140 KB)
    const size_t smem = tfi::tc::leaf_tc32_layout(NB, p->max_leaf32, fts).bytes;
    // persistent: the plan's CTAs, each over its own list of leaves
    dim3 grid(unsigned(p->leaf32_grid), unsigned((d + NB - 1) / NB));
    auto k = fts > 0 ? tfi::tc::leaf_tc32_kernel<NB, true> : tfi::tc::leaf_tc32_kernel<NB, false>;
    k<<<grid, tfi::tc::kL32Threads, smem, s>>>(p->leaf32, p->leaf32_ptr, p->leaf_vtx, p->leaf_dist, p->leaf_pdist, F, d,
                                              p->ftab, fts, p->max_leaf32, lbuf, p->leaf_row, p->hk_err + 1);
}

// returns the number of kernels launched
int launch_leaf_tc32(tfi_plan_t p, const float *F, float *lbuf, int d, cudaStream_t s) {
    if (p->n_leaf32 == 0) return 0;
    if (d <= 16) launch_leaf_tc32_nb<16>(p, F, lbuf, d, s);
    else if (d <= 32) launch_leaf_tc32_nb<32>(p, F, lbuf, d, s);
    else launch_leaf_tc32_nb<64>(p, F, lbuf, d, s);
    return 1;
}

// (a3) bin sums -> kb (the plan's kbuf by default): segments, then the multi-segment bins'
// partial rows in order
template <typename T>
void launch_bucket(tfi_plan_t p, const T *F, int d, cudaStream_t s, float *kb = nullptr) {
    if (!kb) kb = p->kbuf;
    if (d % 4 == 0 && (reinterpret_cast<uintptr_t>(F) % (4 * sizeof(T))) == 0) {
        tfi::dev::bucket_seg_kernel<T, 4><<<grid_for(p->n_segs * (d / 4), 256), 256, 0, s>>>(
            p->n_segs, p->seg_ptr, p->seg_dst, p->key_vtx, F, d, kb, p->sbuf);
        if (p->n_multi > 0)
            tfi::dev::bucket_combine<4><<<grid_for(p->n_multi * (d / 4), 256), 256, 0, s>>>(
                p->n_multi, p->mb_key, p->mb_ptr, d, p->sbuf, kb);
    } else {
        tfi::dev::bucket_seg_kernel<T, 1><<<grid_for(p->n_segs * d, 256), 256, 0, s>>>(
            p->n_segs, p->seg_ptr, p->seg_dst, p->key_vtx, F, d, kb, p->sbuf);
        if (p->n_multi > 0)
            tfi::dev::bucket_combine<1><<<grid_for(p->n_multi * d, 256), 256, 0, s>>>(p->n_multi, p->mb_key,
                                                                                     p->mb_ptr, d, p->sbuf, kb);
    }
}

// (a7) dense leaves -> lbuf: tensor cores for wide BF16 fields and for the big leaves of FP32
// fields with d >= 16 (any d with TFI_PLAN_LEAF_TC), the FP32-ALU kernels for the rest. Below 16
// channels the FP32 ALUs are faster: the f(D) operand costs the same at any d, the ALU sum
// d FMAs per pair (measured at N = 2^20, s0 = 512: 0.34 against 0.21 ms at d = 1, 0.47 against
// 0.48 ms at d = 16, 1.18 against 1.96 ms at d = 64).
// returns the number of kernels launched
template <typename T>
int launch_leaves(tfi_plan_t p, const T *F, int d, cudaStream_t s) {
    const bool alu = (p->hp.flags & TFI_PLAN_LEAF_ALU) != 0;
    if constexpr (sizeof(T) == 2) {
        if (d >= kLeafTcMinChannels && !alu) return launch_leaf_tc(p, F, p->lbuf, d, s);
    }
    bool big = true;
    int launched = 0;
    if constexpr (sizeof(T) == 4) {
        const bool by_default = d >= kLeafTc32MinChannels && p->leaf_share >= kLeafTc32MinShare;
        if (!alu && (by_default || (p->hp.flags & TFI_PLAN_LEAF_TC)) && p->n_leaf32 > 0) {
            launched += launch_leaf_tc32(p, F, p->lbuf, d, s);
            big = false;
        }
    }
    if (d >= 16) launched += launch_leaf<16>(p, F, p->lbuf, d, s, big);
    else if (d > 4) launched += launch_leaf<8>(p, F, p->lbuf, d, s, big);
    else if (d > 2) launched += launch_leaf<4>(p, F, p->lbuf, d, s, big);
    else if (d == 2) launched += launch_leaf<2>(p, F, p->lbuf, d, s, big);
    else launched += launch_leaf<1>(p, F, p->lbuf, d, s, big);
    return launched;
}

// direct jobs of 64 .. 4096 bins on the tensor cores (d > 16, or d = 16 from 512 bins): NB channels
// per CTA
template <int NB>
void launch_table_tc32_nb(tfi_plan_t p, const WorkLists &wl, int d, cudaStream_t s) {
    int fts = wl.tab_fts;
    if (fts > int(p->hp.ftab.size()) ||
        tfi::tc::table_tc32_layout(NB, wl.tab_max_keys, fts).bytes > kLeaf32SmemMax)
        fts = 0;
    // two CTAs per SM by their registers (as for the leaves), no shared-memory padding
    const size_t smem = tfi::tc::table_tc32_layout(NB, wl.tab_max_keys, fts).bytes;
    dim3 grid(unsigned(wl.tab_grid), unsigned((d + NB - 1) / NB));
    auto k = fts > 0 ? tfi::tc::table_tc32_kernel<NB, true> : tfi::tc::table_tc32_kernel<NB, false>;
    k<<<grid, tfi::tc::kL32Threads, smem, s>>>(wl.d_tab, wl.d_tab_ptr, p->key_r, p->key_x, d, p->kbuf, p->vbuf,
                                              p->ftab, fts, wl.tab_max_keys, p->hk_err + 1);
}

void launch_table_tc32(tfi_plan_t p, const WorkLists &wl, int d, cudaStream_t s) {
    if (wl.n_tab == 0) return;
    if (d <= 16) launch_table_tc32_nb<16>(p, wl, d, s);
    else if (d <= 32) launch_table_tc32_nb<32>(p, wl, d, s);
    else launch_table_tc32_nb<64>(p, wl, d, s);
}

template <int CH>
void launch_direct(tfi_plan_t p, const WorkLists &wl, int d, cudaStream_t s) {
    launch_table_tc32(p, wl, d, s);
    if (wl.n_dir == 0) return;
    constexpr int WARPS = 4;
    dim3 grid((wl.n_dir + WARPS - 1) / WARPS, (d + CH - 1) / CH);
    if (CH % 4 == 0 && d % CH == 0)
        tfi::dev::direct_kernel<CH, WARPS, (CH % 4 == 0)><<<grid, 32 * WARPS, 0, s>>>(
            wl.d_dir, wl.n_dir, p->jobs, p->key_r, p->key_x, d, p->kbuf, p->vbuf, p->ftab);
    else
        tfi::dev::direct_kernel<CH, WARPS, false><<<grid, 32 * WARPS, 0, s>>>(wl.d_dir, wl.n_dir, p->jobs, p->key_r,
                                                                              p->key_x, d, p->kbuf, p->vbuf, p->ftab);
}

std::mutex g_attr_mu;
std::atomic<bool> g_attr_done[kMaxDevices] = {};

// Raises the dynamic shared-memory limits of the kernels that need more than 48 KB,
// once per device (the attribute is per device): under a mutex, so that concurrent
// first calls on one device do not race, with a lock-free fast path afterwards.
tfi_status set_attributes() {
    int dev = -1;
    TFI_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(TFI_ERR_ARG, "device ordinal out of range");
    if (g_attr_done[dev].load(std::memory_order_acquire)) return TFI_OK;
    std::lock_guard<std::mutex> lock(g_attr_mu);
    if (g_attr_done[dev].load(std::memory_order_relaxed)) return TFI_OK;
    TFI_CUDA(cudaFuncSetAttribute(tfi::dev::fft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 140 * 1024));
    TFI_CUDA(cudaFuncSetAttribute(tfi::dev::fft_x2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 140 * 1024));
    TFI_CUDA(cudaFuncSetAttribute(tfi::tc::hankel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    TFI_CUDA(cudaFuncSetAttribute(tfi::dev::big_blocks, cudaFuncAttributeMaxDynamicSharedMemorySize, 140 * 1024));
    TFI_CUDA(cudaFuncSetAttribute(tfi::dev::big_columns<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 140 * 1024));
    TFI_CUDA(cudaFuncSetAttribute(tfi::dev::big_columns<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 140 * 1024));
#define LEAF_TC_ATTR(T, NB)                                                                                 \
    TFI_CUDA(cudaFuncSetAttribute(tfi::tc::leaf_tc_kernel<T, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                  227 * 1024));
    LEAF_TC_ATTR(__nv_bfloat16, 64) LEAF_TC_ATTR(__nv_bfloat16, 128) LEAF_TC_ATTR(__nv_bfloat16, 256)
#undef LEAF_TC_ATTR
#define LEAF_TC32_ATTR(NB)                                                                                         \
    TFI_CUDA(cudaFuncSetAttribute(tfi::tc::leaf_tc32_kernel<NB, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                  int(kLeaf32SmemMax)));                                                             \
    TFI_CUDA(cudaFuncSetAttribute(tfi::tc::leaf_tc32_kernel<NB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                  int(kLeaf32SmemMax)));
    LEAF_TC32_ATTR(16) LEAF_TC32_ATTR(32) LEAF_TC32_ATTR(64)
#undef LEAF_TC32_ATTR
#define TABLE_TC32_ATTR(NB)                                                                                         \
    TFI_CUDA(cudaFuncSetAttribute(tfi::tc::table_tc32_kernel<NB, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                  int(kLeaf32SmemMax)));                                                              \
    TFI_CUDA(cudaFuncSetAttribute(tfi::tc::table_tc32_kernel<NB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                  int(kLeaf32SmemMax)));
    TABLE_TC32_ATTR(16) TABLE_TC32_ATTR(32) TABLE_TC32_ATTR(64)
#undef TABLE_TC32_ATTR
#define LEAF_ATTR(T, CH, FS)                                                                                    \
    TFI_CUDA(cudaFuncSetAttribute(tfi::dev::leaf_kernel<T, CH, FS>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                  200 * 1024));
#define LEAF_ATTR2(T, CH) LEAF_ATTR(T, CH, true) LEAF_ATTR(T, CH, false)
    LEAF_ATTR2(float, 1) LEAF_ATTR2(float, 2) LEAF_ATTR2(float, 4) LEAF_ATTR2(float, 8) LEAF_ATTR2(float, 16)
    LEAF_ATTR2(__nv_bfloat16, 1) LEAF_ATTR2(__nv_bfloat16, 2) LEAF_ATTR2(__nv_bfloat16, 4)
    LEAF_ATTR2(__nv_bfloat16, 8) LEAF_ATTR2(__nv_bfloat16, 16)
#undef LEAF_ATTR2
#undef LEAF_ATTR
#define LEAF_WARP_ATTR(T, CH, FS)                                                                                    \
    TFI_CUDA(cudaFuncSetAttribute(tfi::dev::leaf_warp_kernel<T, CH, FS>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                  200 * 1024));
#define LEAF_WARP_ATTR2(T, CH) LEAF_WARP_ATTR(T, CH, true) LEAF_WARP_ATTR(T, CH, false)
    LEAF_WARP_ATTR2(float, 1) LEAF_WARP_ATTR2(float, 2) LEAF_WARP_ATTR2(float, 4) LEAF_WARP_ATTR2(float, 8)
    LEAF_WARP_ATTR2(float, 16) LEAF_WARP_ATTR2(__nv_bfloat16, 1) LEAF_WARP_ATTR2(__nv_bfloat16, 2)
    LEAF_WARP_ATTR2(__nv_bfloat16, 4) LEAF_WARP_ATTR2(__nv_bfloat16, 8) LEAF_WARP_ATTR2(__nv_bfloat16, 16)
#undef LEAF_WARP_ATTR2
#undef LEAF_WARP_ATTR
    g_attr_done[dev].store(true, std::memory_order_release);
    return TFI_OK;
}

// NVTX names of the stages (TFI_STAGE_* order): each stage's launches form one
// range on the host timeline, visible to nsys and usable as an ncu --nvtx filter
// (no cost unless a tool is attached)
const char *const kStageName[] = {"tfi.leaf", "tfi.bucket", "tfi.fft", "tfi.direct", "tfi.gather", "tfi.sweep",
                                  "tfi.hankel"};

struct StageMark {
    tfi_plan_t p;
    cudaStream_t s;
    int stage;
    cudaEvent_t a = nullptr;
    nvtxRangeId_t range = 0;
    bool open = true;
    StageMark(tfi_plan_t p_, cudaStream_t s_, int st) : p(p_), s(s_), stage(st) {
        range = nvtxRangeStartA(kStageName[st]);
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(s, &cs);
        if (p->profiling && cs == cudaStreamCaptureStatusNone && (a = p->next_event())) cudaEventRecord(a, s);
    }
    ~StageMark() {
        if (open) nvtxRangeEnd(range);
    }
    void done(int launches) {
        nvtxRangeEnd(range);
        open = false;
        if (!a) return;
        cudaEvent_t b = p->next_event();
        if (!b) return;
        cudaEventRecord(b, s);
        p->prof.push_back({stage, launches, a, b});
    }
};

void launch_zero_rows(tfi_plan_t p, float *vbuf, int d, cudaStream_t s) {
    const unsigned gy = unsigned(std::min<int32_t>(p->n_zero_ranges, 65535));
    tfi::dev::zero_rows<<<dim3(4, gy), 256, 0, s>>>(p->zero_ranges, p->n_zero_ranges, d, vbuf);
}

template <typename T>
tfi_status apply_impl(tfi_plan_t p, const T *F, T *out, int d, cudaStream_t s) {
    struct ApplyRange {  // the whole apply as one NVTX range
        nvtxRangeId_t id = nvtxRangeStartA("tfi.apply");
        ~ApplyRange() { nvtxRangeEnd(id); }
    } apply_range;
    WorkLists *wl = nullptr;
    if (tfi_status rc = build_work(p, d, &wl)) return rc;
    if (tfi_status rc = set_attributes()) return rc;
    const int n = p->hp.n;
    cudaStream_t s_leaf = p->aux[0], s_dir = p->aux[1], s_crit = p->aux[2];
    if (p->serialize) s_leaf = s_dir = s_crit = s;  // measurement mode: stages one after another
    // fork: everything on the side streams starts after the work already queued on s
    TFI_CUDA(cudaEventRecord(p->ev_fork, s));
    TFI_CUDA(cudaStreamWaitEvent(s_crit, p->ev_fork, 0));
    TFI_CUDA(cudaStreamWaitEvent(s_leaf, p->ev_fork, 0));
    const int64_t n_keys = int64_t(p->hp.key_r.size());
    // (a3) bin sums, first on the high-priority stream
    if (n_keys > 0) {
        StageMark m_bucket(p, s_crit, TFI_STAGE_BUCKET);
        launch_bucket(p, F, d, s_crit);
        m_bucket.done(p->n_multi > 0 ? 2 : 1);
        TFI_CUDA(cudaEventRecord(p->ev_bucket, s_crit));
    }
    // (a7) dense leaves -> lbuf, on the leaf stream; ahead of them, the bins cut from their tables
    // by the support truncation get zero values (no inputs needed; timed with the leaves)
    StageMark m_leaf(p, s_leaf, TFI_STAGE_LEAF);
    int leaf_launches = 0;
    if (p->n_zero_ranges > 0) {
        launch_zero_rows(p, p->vbuf, d, s_leaf);
        ++leaf_launches;
    }
    leaf_launches += launch_leaves(p, F, d, s_leaf);
    m_leaf.done(leaf_launches);
    TFI_CUDA(cudaEventRecord(p->ev_leaf, s_leaf));
    if (n_keys > 0) {
        TFI_CUDA(cudaStreamWaitEvent(s_dir, p->ev_bucket, 0));
        // (a4, a5) tables: direct and Hankel jobs on their stream, sweeps and FFT jobs (one launch per
        // size class) after the bin sums on the critical-path stream
        StageMark m_dir(p, s_dir, TFI_STAGE_DIRECT);
        if (d >= 16) launch_direct<16>(p, *wl, d, s_dir);
        else if (d > 4) launch_direct<8>(p, *wl, d, s_dir);
        else if (d > 2) launch_direct<4>(p, *wl, d, s_dir);
        else if (d == 2) launch_direct<2>(p, *wl, d, s_dir);
        else launch_direct<1>(p, *wl, d, s_dir);
        m_dir.done((wl->n_dir > 0 ? 1 : 0) + (wl->n_tab > 0 ? 1 : 0));
        if (wl->n_hk > 0) {
            StageMark m_hk(p, s_dir, TFI_STAGE_HANKEL);
            tfi::tc::hankel_kernel<<<wl->n_hk, 128, wl->hk_smem, s_dir>>>(wl->d_hk, p->key_r, p->key_x, d, p->kbuf,
                                                                          p->vbuf, p->ftab, p->hk_err);
            m_hk.done(1);
        }
        TFI_CUDA(cudaEventRecord(p->ev_dir, s_dir));
        if (p->n_sweeps > 0 || p->n_sw_ejobs > 0) {
            StageMark m_sw(p, s_crit, TFI_STAGE_SWEEP);
            constexpr int WARPS = 4;
            const unsigned cblocks = unsigned((d + tfi::dev::kSweepCH - 1) / tfi::dev::kSweepCH);
            if (p->n_sweeps > 0)
                tfi::dev::sweep_g_kernel<WARPS>
                    <<<dim3(unsigned((p->n_sweeps + WARPS - 1) / WARPS), cblocks), 32 * WARPS, 0, s_crit>>>(
                        p->sw_jobs, p->n_sweeps, p->key_r, p->key_x, p->sw_keys, p->sw_run, d, p->kbuf, p->vbuf,
                        p->sw_scratch, p->sw_beta, p->sw_coef, p->sw_terms);
            if (p->n_sw_ejobs > 0)
                tfi::dev::sweep_e_kernel<WARPS>
                    <<<dim3(unsigned((p->n_sw_ejobs + WARPS - 1) / WARPS), cblocks), 32 * WARPS, 0, s_crit>>>(
                        p->sw_ejobs, p->n_sw_ejobs, p->jobs, p->key_r, d, p->kbuf, p->vbuf, p->sw_beta, p->sw_coef,
                        p->sw_terms);
            m_sw.done((p->n_sweeps > 0) + (p->n_sw_ejobs > 0));
        }
        StageMark m_fft(p, s_crit, TFI_STAGE_FFT);
        for (size_t c = 0; c < wl->fft_lnp.size(); ++c) {
            const int np = wl->fft_npair[c];
            if (np >= 2) {
                // two channel pairs per shared-memory element
                const size_t smem = size_t((np + 1) / 2) * (size_t(1) << wl->fft_lnp[c]) * sizeof(ulonglong2);
                tfi::dev::fft_x2_kernel<<<wl->fft_count[c], kFftThreads, smem, s_crit>>>(
                    wl->d_fft + wl->fft_off[c], p->jobs, p->key_r, p->key_x, d, p->kbuf, p->vbuf, p->spectra,
                    p->twiddle, reinterpret_cast<const ulonglong2 *>(p->twiddle_b));
            } else {
                const size_t smem = size_t(np) * size_t(tfi::dev::padded_size(1 << wl->fft_lnp[c])) * sizeof(float2);
                tfi::dev::fft_kernel<<<wl->fft_count[c], kFftThreads, smem, s_crit>>>(
                    wl->d_fft + wl->fft_off[c], p->jobs, p->key_r, p->key_x, d, p->kbuf, p->vbuf, p->spectra,
                    p->twiddle);
            }
        }
        launch_big(p, *wl, d, s_crit);
        m_fft.done(int(wl->fft_lnp.size()) + big_launches(*wl));
        TFI_CUDA(cudaEventRecord(p->ev_crit, s_crit));
        TFI_CUDA(cudaStreamWaitEvent(s, p->ev_crit, 0));
        TFI_CUDA(cudaStreamWaitEvent(s, p->ev_dir, 0));
    } else {
        // nothing on the critical-path stream: join it so that it holds no dangling fork
        TFI_CUDA(cudaEventRecord(p->ev_crit, s_crit));
        TFI_CUDA(cudaStreamWaitEvent(s, p->ev_crit, 0));
    }
    // join, then (a6) gather
    TFI_CUDA(cudaStreamWaitEvent(s, p->ev_leaf, 0));
    StageMark m_gather(p, s, TFI_STAGE_GATHER);
    if (d % 4 == 0 && (reinterpret_cast<uintptr_t>(out) % (4 * sizeof(T))) == 0)
        tfi::dev::gather_kernel<T, 4><<<grid_for(int64_t(n) * (d / 4), 256), 256, 0, s>>>(
            n, p->gorder, p->vrec_ptr, p->vrec_akey, p->vrec_bkey, p->vbuf, p->lbuf, p->in_leaf, d, out);
    else
        tfi::dev::gather_kernel<T, 1><<<grid_for(int64_t(n) * d, 256), 256, 0, s>>>(
            n, p->gorder, p->vrec_ptr, p->vrec_akey, p->vrec_bkey, p->vbuf, p->lbuf, p->in_leaf, d, out);
    m_gather.done(1);
    TFI_CUDA(cudaGetLastError());
    return TFI_OK;
}

// Device allocations that live for one plan-time pass.
struct DeviceTemps {
    std::vector<void *> ptrs;
    ~DeviceTemps() {
        for (void *q : ptrs) cudaFree(q);
    }
    template <typename T>
    tfi_status get(T **dst, size_t count) {
        void *q = nullptr;
        if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) return fail(TFI_ERR_OOM, "cudaMalloc failed (device keys)");
        ptrs.push_back(q);
        *dst = static_cast<T *>(q);
        return TFI_OK;
    }
};

// (a2) device distances and bin keys at plan time; temporaries are freed here.
tfi_status run_device_keys(tfi_plan_t p) {
    const tfi::HostPlan &hp = p->hp;
    const int n = hp.n;
    const int64_t R = int64_t(hp.recs.size());
    if (R == 0) return TFI_OK;
    DeviceTemps tmp;
    int K = 1;
    while ((1 << K) <= hp.k1_maxhop) ++K;  // 2^K > largest hop depth
    int32_t *parent, *qpar, *rv, *ra, *rp, *hop0, *hop1, *anc;
    int64_t *D0, *D1;
    if (tfi_status rc = tmp.get(&parent, size_t(n))) return rc;
    if (tfi_status rc = tmp.get(&qpar, size_t(n))) return rc;
    if (tfi_status rc = tmp.get(&rv, size_t(R))) return rc;
    if (tfi_status rc = tmp.get(&ra, size_t(R))) return rc;
    if (tfi_status rc = tmp.get(&rp, size_t(R))) return rc;
    if (tfi_status rc = tmp.get(&hop0, size_t(n))) return rc;
    if (tfi_status rc = tmp.get(&hop1, size_t(n))) return rc;
    if (tfi_status rc = tmp.get(&D0, size_t(n))) return rc;
    if (tfi_status rc = tmp.get(&D1, size_t(n))) return rc;
    if (tfi_status rc = tmp.get(&anc, size_t(K + 1) * size_t(n))) return rc;
    std::vector<int32_t> rec_v(static_cast<size_t>(R));
    for (int64_t i = 0; i < R; ++i) rec_v[size_t(i)] = hp.recs[size_t(i)].v;
    TFI_CUDA(cudaMemcpy(parent, hp.k1_parent.data(), size_t(n) * 4, cudaMemcpyHostToDevice));
    TFI_CUDA(cudaMemcpy(qpar, hp.k1_qpar.data(), size_t(n) * 4, cudaMemcpyHostToDevice));
    TFI_CUDA(cudaMemcpy(rv, rec_v.data(), size_t(R) * 4, cudaMemcpyHostToDevice));
    TFI_CUDA(cudaMemcpy(ra, hp.rec_anchor.data(), size_t(R) * 4, cudaMemcpyHostToDevice));
    TFI_CUDA(cudaMemcpy(rp, hp.rec_p1.data(), size_t(R) * 4, cudaMemcpyHostToDevice));
    void *outr = nullptr, *outx = nullptr;
    if (tfi_status rc = p->alloc(&outr, size_t(R) * 4)) return rc;
    if (tfi_status rc = p->alloc(&outx, size_t(R) * 4)) return rc;
    p->dev_rec_r = static_cast<int32_t *>(outr);
    p->dev_rec_x = static_cast<int32_t *>(outx);
    cudaEvent_t e0, e1;
    TFI_CUDA(cudaEventCreate(&e0));
    TFI_CUDA(cudaEventCreate(&e1));
    TFI_CUDA(cudaEventRecord(e0, 0));
    const int gb = grid_for(n, 256);
    tfi::dev::k1_init<<<gb, 256>>>(n, parent, qpar, D0, hop0, anc);
    for (int k = 0; k < K; ++k) {
        tfi::dev::k1_jump<<<gb, 256>>>(n, anc + int64_t(k) * n, D0, hop0, anc + int64_t(k + 1) * n, D1, hop1);
        std::swap(D0, D1);
        std::swap(hop0, hop1);
    }
    tfi::dev::k1_records<<<grid_for(R, 256), 256>>>(R, rv, ra, rp, D0, hop0, anc, n, K, p->dev_rec_r, p->dev_rec_x);
    TFI_CUDA(cudaGetLastError());
    TFI_CUDA(cudaEventRecord(e1, 0));
    TFI_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    p->device_keys_ms = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return TFI_OK;
}

// The dense leaves in launch form: runs of consecutive leaves of fewer than
// kLeafWarpMin vertices in groups of at most kLeafGroup vertices, as [begin, end)
// pairs of leaf_vtx positions (a big leaf ends the run before it), and the big
// leaves' ranges in plan order.
void split_leaves(const tfi::HostPlan &hp, std::vector<int32_t> &sgrp, std::vector<int32_t> &big_lo,
                  std::vector<int32_t> &big_hi) {
    const int32_t nl = int32_t(hp.leaf_vtx.size());
    int32_t gb = -1;
    for (int32_t pos = 0; pos < nl;) {
        const int32_t lo = hp.leaf_lo[size_t(pos)], hi = hp.leaf_hi[size_t(pos)];
        if (hi - lo >= tfi::dev::kLeafWarpMin) {
            if (gb >= 0) sgrp.insert(sgrp.end(), {gb, lo});
            gb = -1;
            big_lo.push_back(lo);
            big_hi.push_back(hi);
        } else if (gb < 0) {
            gb = lo;
        } else if (hi - gb > tfi::kLeafGroup) {
            sgrp.insert(sgrp.end(), {gb, lo});
            gb = lo;
        }
        pos = hi;
    }
    if (gb >= 0) sgrp.insert(sgrp.end(), {gb, nl});
}

// FP32 tensor-core leaves: every leaf of >= kLeafWarpMin vertices as [lo, hi) (from split_leaves),
// sorted largest first, then dealt to min(leaves, ctas_cap) persistent CTAs longest first
// (lpt_schedule): `grouped` CTA by CTA, `ptr` the CTA offsets; returns the CTA count.
int leaf32_schedule(const std::vector<int32_t> &big_lo, const std::vector<int32_t> &big_hi, int ctas_cap,
                    std::vector<int2> &grouped, std::vector<int32_t> &ptr, int32_t *max_leaf) {
    std::vector<int2> l32;
    for (size_t q = 0; q < big_lo.size(); ++q) {
        l32.push_back(make_int2(big_lo[q], big_hi[q]));
        *max_leaf = std::max(*max_leaf, big_hi[q] - big_lo[q]);
    }
    std::stable_sort(l32.begin(), l32.end(), [](int2 a, int2 b) { return a.y - a.x > b.y - b.x; });
    const int ctas = std::min(int(l32.size()), ctas_cap);
    lpt_schedule(l32, ctas, [](int2 a) { return a.y - a.x; }, grouped, ptr);
    return ctas;
}

// Depth-first preorder of the forest, tree by tree from the smallest unvisited
// vertex: the order in which the gather takes the vertices.
std::vector<int32_t> depth_first_order(const tfi::HostPlan &hp) {
    std::vector<int32_t> order;
    order.reserve(size_t(hp.n));
    std::vector<uint8_t> seen(size_t(hp.n), 0);
    std::vector<int32_t> stack;
    for (int32_t r = 0; r < hp.n; ++r) {
        if (seen[size_t(r)]) continue;
        seen[size_t(r)] = 1;
        stack.push_back(r);
        while (!stack.empty()) {
            const int32_t v = stack.back();
            stack.pop_back();
            order.push_back(v);
            for (int64_t e = hp.ptr[size_t(v)]; e < hp.ptr[size_t(v) + 1]; ++e) {
                const int32_t w = hp.adj[size_t(e)];
                if (!seen[size_t(w)]) {
                    seen[size_t(w)] = 1;
                    stack.push_back(w);
                }
            }
        }
    }
    return order;
}

// interleaved complex values (re, im, re, im, ...) -> one (re, re, im, im) per value, the
// operand form of the paired FP32 instructions in fft_x2_kernel
std::vector<float4> broadcast_pairs(const std::vector<float> &z) {
    std::vector<float4> out(z.size() / 2);
    for (size_t i = 0; i < out.size(); ++i) out[i] = make_float4(z[2 * i], z[2 * i], z[2 * i + 1], z[2 * i + 1]);
    return out;
}

tfi_status upload_plan(tfi_plan_t p) {
    tfi::HostPlan &hp = p->hp;
    TFI_CUDA(cudaGetDevice(&p->device));
    if (tfi_status rc = p->upload(&p->key_r, hp.key_r)) return rc;
    if (tfi_status rc = p->upload(&p->key_x, hp.key_x)) return rc;
    if (tfi_status rc = p->upload(&p->key_ptr, hp.key_ptr)) return rc;
    if (tfi_status rc = p->upload(&p->key_vtx, hp.key_vtx)) return rc;
    std::vector<tfi::dev::JobDev> jd(hp.jobs.size());
    for (size_t j = 0; j < hp.jobs.size(); ++j) {
        const tfi::Job &jb = hp.jobs[j];
        jd[j].kb = int32_t(jb.kb);
        jd[j].ke = int32_t(jb.ke);
        jd[j].lp1 = jb.lp1;
        jd[j].lp2 = jb.lp2;
        jd[j].spec_off = jb.mode == 0 ? int32_t(hp.spec_class_off[size_t(jb.lp1 * 32 + jb.lp2)] / 2) : 0;
        jd[j].pad = 0;
    }
    if (tfi_status rc = p->upload(&p->jobs, jd)) return rc;
    {
        std::vector<tfi::dev::DirItem> dir;
        std::map<int, std::vector<int32_t>> by_class;
        for (size_t j = 0; j < hp.jobs.size(); ++j) {
            const tfi::Job &jb = hp.jobs[j];
            if (jb.ke == jb.kb || jb.mode == 2 || jb.mode == 3 || jb.mode == 4) continue;
            if (jb.mode == 0) {
                by_class[jb.lp1 + jb.lp2].push_back(int32_t(j));
            } else {
                for (int64_t q = jb.kb; q < jb.ke; q += 64) dir.push_back(tfi::dev::DirItem{int32_t(j), int32_t(q)});
            }
        }
        std::vector<int32_t> fj;
        for (auto &kv : by_class) {
            p->st_cls_lnp.push_back(kv.first);
            p->st_cls_joff.push_back(int32_t(fj.size()));
            p->st_cls_njobs.push_back(int32_t(kv.second.size()));
            fj.insert(fj.end(), kv.second.begin(), kv.second.end());
        }
        if (tfi_status rc = p->upload(&p->st_dir, dir)) return rc;
        if (tfi_status rc = p->upload(&p->st_fft_job, fj)) return rc;
        p->n_st_dir = int32_t(dir.size());
    }
    p->n_hankel = 0;
    for (const tfi::Job &jb : hp.jobs) p->n_hankel += jb.mode == 3;
    p->n_big_jobs = 0;
    for (const tfi::Job &jb : hp.jobs) p->n_big_jobs += jb.mode == 4;
    if (tfi_status rc = p->upload(&p->zero_ranges, hp.zero_ranges)) return rc;
    p->n_zero_ranges = int32_t(hp.zero_ranges.size() / 2);
    if (p->n_big_jobs > 0) {
        std::vector<float2> hi(8192), lo(8192);
        for (int j = 0; j < 8192; ++j) {
            const double a = -2.0 * M_PI * double(j) / 8192.0, b = -2.0 * M_PI * double(j) / double(1 << 26);
            hi[size_t(j)] = make_float2(float(std::cos(a)), float(std::sin(a)));
            lo[size_t(j)] = make_float2(float(std::cos(b)), float(std::sin(b)));
        }
        if (tfi_status rc = p->upload(&p->big_tw_hi, hi)) return rc;
        if (tfi_status rc = p->upload(&p->big_tw_lo, lo)) return rc;
    }
    {
        void *q = nullptr;
        if (tfi_status rc = p->alloc(&q, 16)) return rc;
        p->hk_err = static_cast<int32_t *>(q);
        TFI_CUDA(cudaMemset(p->hk_err, 0, 16));
    }
    if (tfi_status rc = p->upload(&p->lgrp_ptr, hp.lgrp_ptr)) return rc;
    if (tfi_status rc = p->upload(&p->leaf_vtx, hp.leaf_vtx)) return rc;
    if (tfi_status rc = p->upload(&p->leaf_dist, hp.leaf_dist)) return rc;
    if (tfi_status rc = p->upload(&p->leaf_pdist, hp.leaf_pdist)) return rc;
    if (tfi_status rc = p->upload(&p->leaf_lo, hp.leaf_lo)) return rc;
    if (tfi_status rc = p->upload(&p->leaf_hi, hp.leaf_hi)) return rc;
    {
        const std::vector<int32_t> order = depth_first_order(hp);
        if (tfi_status rc = p->upload(&p->gorder, order)) return rc;
        // the gather's record lists in its own vertex order: the threads of a warp, at
        // consecutive positions, read consecutive (A-key, b-key) entries
        std::vector<int32_t> gptr(size_t(hp.n) + 1, 0), gak, gbk;
        gak.reserve(hp.vrec_akey.size());
        gbk.reserve(hp.vrec_bkey.size());
        for (size_t i = 0; i < order.size(); ++i) {
            const size_t u = size_t(order[i]);
            for (int32_t e = hp.vrec_ptr[u]; e < hp.vrec_ptr[u + 1]; ++e) {
                gak.push_back(hp.vrec_akey[size_t(e)]);
                gbk.push_back(hp.vrec_bkey[size_t(e)]);
            }
            gptr[i + 1] = int32_t(gak.size());
        }
        if (tfi_status rc = p->upload(&p->vrec_ptr, gptr)) return rc;
        if (tfi_status rc = p->upload(&p->vrec_akey, gak)) return rc;
        if (tfi_status rc = p->upload(&p->vrec_bkey, gbk)) return rc;
        // leaf terms in the same order: the leaf kernels write the row of a vertex at its gather
        // position, so the gather reads them in sequence
        std::vector<int32_t> pos(size_t(hp.n), 0);
        for (size_t i = 0; i < order.size(); ++i) pos[size_t(order[i])] = int32_t(i);
        std::vector<int32_t> lrow(hp.leaf_vtx.size());
        for (size_t j = 0; j < lrow.size(); ++j) lrow[j] = pos[size_t(hp.leaf_vtx[j])];
        std::vector<uint8_t> inl(size_t(hp.n), 0);
        for (size_t i = 0; i < order.size(); ++i) inl[i] = hp.in_leaf[size_t(order[i])];
        if (tfi_status rc = p->upload(&p->leaf_row, lrow)) return rc;
        if (tfi_status rc = p->upload(&p->in_leaf, inl)) return rc;
    }
    p->n_groups = int32_t(hp.lgrp_ptr.size()) - 1;
    {
        std::vector<int32_t> sgrp, leaf_lo_big, leaf_hi_big;
        split_leaves(hp, sgrp, leaf_lo_big, leaf_hi_big);
        for (size_t q = 0; q < sgrp.size(); q += 2) p->max_sgs = std::max(p->max_sgs, sgrp[q + 1] - sgrp[q]);
        p->n_sgroups = int32_t(sgrp.size() / 2);
        std::vector<int32_t> bptr, blo, bhi;
        pack_big_leaves(leaf_lo_big, leaf_hi_big, bptr, blo, bhi, &p->max_big);
        p->n_big = int32_t(bptr.size()) - 1;
        if (tfi_status rc = p->upload(&p->big_ptr, bptr)) return rc;
        if (tfi_status rc = p->upload(&p->sgrp_ptr, sgrp)) return rc;
        if (tfi_status rc = p->upload(&p->big_lo, blo)) return rc;
        if (tfi_status rc = p->upload(&p->big_hi, bhi)) return rc;
        // FP32 tensor-core leaves: every big leaf, dealt longest first to persistent CTAs, two per
        // SM (their tensor memory)
        std::vector<int2> grouped;
        std::vector<int32_t> ptr;
        p->leaf32_grid = leaf32_schedule(leaf_lo_big, leaf_hi_big, 2 * device_sms(), grouped, ptr, &p->max_leaf32);
        p->n_leaf32 = int32_t(grouped.size());
        if (tfi_status rc = p->upload(&p->leaf32, grouped)) return rc;
        if (tfi_status rc = p->upload(&p->leaf32_ptr, ptr)) return rc;
        // per-channel flops: leaf pairs 2 n^2, FFT tables 5 P log2 P + 3 P per channel, direct 2 nk^2
        double leaf = 0, tables = 0;
        for (const tfi::Leaf &l : hp.leaves) leaf += 2.0 * double(l.end - l.begin) * double(l.end - l.begin);
        for (const tfi::Job &j : hp.jobs) {
            const double nk = double(j.ke - j.kb), np = std::ldexp(1.0, j.lp1 + j.lp2);
            if (j.mode == 0 || j.mode == 4) tables += 5.0 * np * double(j.lp1 + j.lp2) + 3.0 * np;
            else if (j.mode == 1) tables += 2.0 * nk * nk;
        }
        p->leaf_share = leaf + tables > 0 ? leaf / (leaf + tables) : 0.0;
    }

    {
        std::vector<tfi::tc::LeafTile> lt;
        for (int g = 0; g < p->n_groups; ++g)
            for (int32_t i0 = hp.lgrp_ptr[size_t(g)]; i0 < hp.lgrp_ptr[size_t(g) + 1]; i0 += tfi::tc::kLeafTile)
                lt.push_back(tfi::tc::LeafTile{hp.lgrp_ptr[size_t(g)], hp.lgrp_ptr[size_t(g) + 1], i0, 0});
        if (tfi_status rc = p->upload(&p->leaf_tiles, lt)) return rc;
        p->n_leaf_tiles = int32_t(lt.size());
    }
    p->max_gs = 1;
    for (int g = 0; g < p->n_groups; ++g)
        p->max_gs = std::max(p->max_gs, hp.lgrp_ptr[size_t(g) + 1] - hp.lgrp_ptr[size_t(g)]);
    if (tfi_status rc = p->upload(&p->ftab, hp.ftab)) return rc;
    std::vector<int32_t> ej;  // component corrections evaluated by the sweeps
    for (size_t j = 0; j < hp.jobs.size(); ++j)
        if (hp.jobs[j].is_comp && hp.jobs[j].mode == 2 && hp.jobs[j].ke > hp.jobs[j].kb) ej.push_back(int32_t(j));
    if (!hp.sweeps.empty() || !ej.empty()) {
        if (hp.sw_beta.empty()) return fail(TFI_ERR_ARG, "exponential-sweep plan without exponential terms");
        std::vector<tfi::dev::SweepJobDev> sj(hp.sweeps.size());
        for (size_t i = 0; i < sj.size(); ++i) {
            const tfi::SweepJob &q = hp.sweeps[i];
            sj[i] = tfi::dev::SweepJobDev{q.sb, q.se, q.rb, q.m, q.cjb, q.cje};
        }
        if (tfi_status rc = p->upload(&p->sw_jobs, sj)) return rc;
        if (tfi_status rc = p->upload(&p->sw_keys, hp.sw_keys)) return rc;
        if (tfi_status rc = p->upload(&p->sw_run, hp.sw_run)) return rc;
        if (tfi_status rc = p->upload(&p->sw_ejobs, ej)) return rc;
        if (tfi_status rc = p->upload(&p->sw_beta, hp.sw_beta)) return rc;
        if (tfi_status rc = p->upload(&p->sw_coef, hp.sw_coef)) return rc;
        void *q = nullptr;
        if (tfi_status rc = p->alloc(&q, std::max<size_t>(hp.sw_run.size(), 1) * 2 * size_t(hp.max_channels) * 4))
            return rc;
        p->sw_scratch = static_cast<float *>(q);
        p->n_sweeps = int32_t(sj.size());
        p->n_sw_ejobs = int32_t(ej.size());
        p->sw_terms = int32_t(hp.sw_beta.size());
    }
    std::vector<float2> spec(hp.spectra.size() / 2), tw(hp.twiddle.size() / 2);
    std::memcpy(spec.data(), hp.spectra.data(), hp.spectra.size() * sizeof(float));
    std::memcpy(tw.data(), hp.twiddle.data(), hp.twiddle.size() * sizeof(float));
    if (tfi_status rc = p->upload(&p->spectra, spec)) return rc;
    if (tfi_status rc = p->upload(&p->twiddle, tw)) return rc;
    if (tfi_status rc = p->upload(&p->twiddle_b, broadcast_pairs(hp.twiddle))) return rc;
    const size_t K = hp.key_r.size(), dm = size_t(hp.max_channels);
    {
        // segments of at most kBucketSeg consecutive members per bin
        std::vector<int32_t> seg_ptr, seg_dst, mb_key, mb_ptr;
        int32_t slots = 0;
        for (size_t k = 0; k < K; ++k) {
            const int32_t b = hp.key_ptr[k], e = hp.key_ptr[k + 1];
            const int32_t ns = std::max<int32_t>(1, (e - b + kBucketSeg - 1) / kBucketSeg);
            if (ns == 1) {
                seg_ptr.push_back(b);
                seg_dst.push_back(int32_t(k));
                continue;
            }
            mb_key.push_back(int32_t(k));
            mb_ptr.push_back(slots);
            for (int32_t q = 0; q < ns; ++q) {
                seg_ptr.push_back(b + q * kBucketSeg);
                seg_dst.push_back(-1 - slots++);
            }
        }
        seg_ptr.push_back(hp.key_ptr[K]);
        mb_ptr.push_back(slots);
        p->n_segs = int64_t(seg_dst.size());
        p->n_multi = int64_t(mb_key.size());
        if (tfi_status rc = p->upload(&p->seg_ptr, seg_ptr)) return rc;
        if (tfi_status rc = p->upload(&p->seg_dst, seg_dst)) return rc;
        if (tfi_status rc = p->upload(&p->mb_key, mb_key)) return rc;
        if (tfi_status rc = p->upload(&p->mb_ptr, mb_ptr)) return rc;
        if (tfi_status rc = p->alloc(reinterpret_cast<void **>(&p->sbuf), size_t(slots) * dm * sizeof(float)))
            return rc;
    }
    if (tfi_status rc = p->alloc(reinterpret_cast<void **>(&p->kbuf), K * dm * sizeof(float))) return rc;
    if (tfi_status rc = p->alloc(reinterpret_cast<void **>(&p->vbuf), K * dm * sizeof(float))) return rc;
    if (tfi_status rc = p->alloc(reinterpret_cast<void **>(&p->lbuf), size_t(hp.n) * dm * sizeof(float))) return rc;
    if (tfi_status rc = run_device_keys(p)) return rc;
    {
        // internal streams above the caller's default priority; the bin sums are queued before the
        // leaves so that their CTAs are dispatched first
        int least = 0, greatest = 0;
        TFI_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        TFI_CUDA(cudaStreamCreateWithPriority(&p->aux[0], cudaStreamNonBlocking, greatest));
        TFI_CUDA(cudaStreamCreateWithPriority(&p->aux[1], cudaStreamNonBlocking, greatest));
        TFI_CUDA(cudaStreamCreateWithPriority(&p->aux[2], cudaStreamNonBlocking, greatest));
    }
    for (cudaEvent_t *e : {&p->ev_fork, &p->ev_leaf, &p->ev_bucket, &p->ev_dir, &p->ev_crit})
        TFI_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    p->on_device = true;
    return TFI_OK;
}

tfi_status check_apply_args(tfi_plan_t p, const void *a, const void *b, int32_t d, int32_t dtype) {
    if (!p || !a || !b) return fail(TFI_ERR_ARG, "null plan or field pointer");
    if (!p->on_device) return fail(TFI_ERR_NO_DEVICE, "plan was built host-only");
    if (d < 1 || d > p->hp.max_channels) return fail(TFI_ERR_ARG, "d must be in [1, max_channels]");
    if (dtype != TFI_DTYPE_F32 && dtype != TFI_DTYPE_BF16) return fail(TFI_ERR_ARG, "unknown dtype");
    if (a == b) return fail(TFI_ERR_ARG, "out must not alias F");
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != p->device)
        return fail(TFI_ERR_ARG, "the current device is not the plan's device");
    return TFI_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free apply (tfi_apply_static): the workspace and the per-d work
// lists live in one file-scope device array instead of plan-owned cudaMalloc
// memory. Every GPU that loads this library holds the array until exit.
// ---------------------------------------------------------------------------
constexpr size_t kStaticScratchBytes = size_t(TFI_STATIC_SCRATCH_BYTES);
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void *g_static_addr[kMaxDevices] = {};

// Device address of g_static_scratch on device `dev` (which must be current).
// In host code the symbol names a host-side stand-in, so the address is looked
// up once per device with cudaGetSymbolAddress and cached.
tfi_status static_scratch_address(int dev, unsigned char **out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(TFI_ERR_ARG, "device ordinal out of range for the static workspace");
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess || !ptr)
            return fail(TFI_ERR_CUDA, std::string("cudaGetSymbolAddress(static workspace): ") + cudaGetErrorString(e));
        g_static_addr[dev] = ptr;
    }
    *out = static_cast<unsigned char *>(g_static_addr[dev]);
    return TFI_OK;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// FFT work items of one size class for tfi_apply_static: job list entry i / per, channel
// pairs (i % per) * np ... of at most np pairs, for `pairs` channel pairs in all.
__global__ void expand_fft_items(const int32_t *__restrict__ job, int n_jobs, int per, int np, int pairs,
                                 tfi::dev::FftItem *__restrict__ items) {
    const int64_t total = int64_t(n_jobs) * per;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int j = int(i / per), r = int(i - int64_t(j) * per);
        items[i] = tfi::dev::FftItem{job[j], r * np, min(np, pairs - r * np)};
    }
}

template <typename T>
tfi_status apply_static_impl(tfi_plan_t p, const T *F, T *out, int d, cudaStream_t s) {
    if (p->n_sweeps > 0 || p->n_sw_ejobs > 0)
        return fail(TFI_ERR_UNSUPPORTED, "tfi_apply_static does not run exponential-sweep plans");
    if (p->n_hankel > 0) return fail(TFI_ERR_UNSUPPORTED, "tfi_apply_static does not run Hankel-evaluator plans");
    if (p->n_big_jobs > 0)
        return fail(TFI_ERR_UNSUPPORTED, "tfi_apply_static does not run plans with four-step FFT tables");
    if (tfi_status rc = set_attributes()) return rc;
    // FFT items for this d: per size class, one item per (job, block of np channel pairs),
    // written into the static array by expand_fft_items (no host-sourced copy)
    const int pairs = (d + 1) / 2;
    const size_t n_cls = p->st_cls_lnp.size();
    std::vector<int> cls_np(n_cls), cls_per(n_cls);
    std::vector<int64_t> cls_off(n_cls);
    int64_t n_fft = 0;
    for (size_t c = 0; c < n_cls; ++c) {
        cls_np[c] = fft_pairs_per_cta(p->st_cls_lnp[c], pairs, kFftSmemPairPoints);
        cls_per[c] = (pairs + cls_np[c] - 1) / cls_np[c];
        cls_off[c] = n_fft;
        n_fft += int64_t(p->st_cls_njobs[c]) * cls_per[c];
    }
    // carve the static array: bin sums, table values, leaf terms, FFT items
    const size_t K = p->hp.key_r.size(), n = size_t(p->hp.n);
    const size_t o_k = 0;
    const size_t o_v = o_k + align256(K * size_t(d) * sizeof(float));
    const size_t o_l = o_v + align256(K * size_t(d) * sizeof(float));
    const size_t o_f = o_l + align256(n * size_t(d) * sizeof(float));
    const size_t total = o_f + align256(size_t(n_fft) * sizeof(tfi::dev::FftItem));
    if (total > kStaticScratchBytes)
        return fail(TFI_ERR_ARG, "plan needs " + std::to_string(total) + " bytes of workspace at d=" + std::to_string(d) +
                                     ", more than the static workspace of " + std::to_string(kStaticScratchBytes) +
                                     " bytes; use tfi_apply");
    unsigned char *base = nullptr;
    if (tfi_status rc = static_scratch_address(p->device, &base)) return rc;
    float *kbuf = reinterpret_cast<float *>(base + o_k);
    float *vbuf = reinterpret_cast<float *>(base + o_v);
    float *lbuf = reinterpret_cast<float *>(base + o_l);
    auto *d_fft = reinterpret_cast<tfi::dev::FftItem *>(base + o_f);
    // every workspace value an apply reads is written earlier in the same apply,
    // so nothing needs clearing between calls
    if (p->n_zero_ranges > 0) launch_zero_rows(p, vbuf, d, s);
    if (p->n_groups > 0) launch_leaf<16>(p, F, lbuf, d, s);
    if (K > 0) {
        tfi::dev::bucket_kernel<T, 1><<<grid_for(int64_t(K) * d, 256), 256, 0, s>>>(int64_t(K), p->key_ptr, p->key_vtx,
                                                                                   F, d, kbuf);
        for (size_t c = 0; c < n_cls; ++c) {
            const int64_t cnt = int64_t(p->st_cls_njobs[c]) * cls_per[c];
            expand_fft_items<<<grid_for(cnt, 256), 256, 0, s>>>(p->st_fft_job + p->st_cls_joff[c], p->st_cls_njobs[c],
                                                                cls_per[c], cls_np[c], pairs, d_fft + cls_off[c]);
            const size_t smem =
                size_t(cls_np[c]) * size_t(tfi::dev::padded_size(1 << p->st_cls_lnp[c])) * sizeof(float2);
            tfi::dev::fft_kernel<<<unsigned(cnt), kFftThreads, smem, s>>>(d_fft + cls_off[c], p->jobs, p->key_r,
                                                                          p->key_x, d, kbuf, vbuf, p->spectra,
                                                                          p->twiddle);
        }
        if (p->n_st_dir > 0) {
            constexpr int WARPS = 4;
            dim3 grid((unsigned(p->n_st_dir) + WARPS - 1) / WARPS, (d + 15) / 16);
            tfi::dev::direct_kernel<16, WARPS, false><<<grid, 32 * WARPS, 0, s>>>(p->st_dir, p->n_st_dir, p->jobs,
                                                                                  p->key_r, p->key_x, d, kbuf, vbuf,
                                                                                  p->ftab);
        }
    }
    tfi::dev::gather_kernel<T, 1><<<grid_for(int64_t(n) * d, 256), 256, 0, s>>>(
        int(n), p->gorder, p->vrec_ptr, p->vrec_akey, p->vrec_bkey, vbuf, lbuf, p->in_leaf, d, out);
    TFI_CUDA(cudaGetLastError());
    return TFI_OK;
}

// ---------------------------------------------------------------------------
// dense tensor-core evaluation
// ---------------------------------------------------------------------------
tfi_status build_dense(tfi_plan_t p) {
    if (p->dense_ready) return TFI_OK;
    const tfi::HostPlan &hp = p->hp;
    const int n = hp.n;
    std::vector<int32_t> vtx, dist, pdist, tree_ptr(1, 0);
    vtx.reserve(size_t(n));
    dist.reserve(size_t(n));
    pdist.reserve(size_t(n));
    std::vector<char> seen(size_t(n), 0);
    std::vector<int64_t> dd(size_t(n), 0);
    std::vector<int32_t> stack, kids;
    int64_t max_diam = 0;
    int32_t max_tree = 1;
    for (int32_t r = 0; r < n; ++r) {
        if (seen[size_t(r)]) continue;
        // preorder from the tree's smallest vertex, children ascending
        const size_t start = vtx.size();
        stack.assign(1, r);
        seen[size_t(r)] = 1;
        dd[size_t(r)] = 0;
        std::vector<int64_t> par_d;
        std::vector<int32_t> order_par;
        while (!stack.empty()) {
            const int32_t v = stack.back();
            stack.pop_back();
            vtx.push_back(v);
            dist.push_back(int32_t(std::min<int64_t>(dd[size_t(v)], INT32_MAX)));
            kids.clear();
            for (int64_t e = hp.ptr[size_t(v)]; e < hp.ptr[size_t(v) + 1]; ++e) {
                const int32_t b = hp.adj[size_t(e)];
                if (seen[size_t(b)]) continue;
                seen[size_t(b)] = 1;
                dd[size_t(b)] = dd[size_t(v)] + hp.qlen[size_t(e)];
                kids.push_back(b);
            }
            for (size_t k = kids.size(); k-- > 0;) stack.push_back(kids[k]);
        }
        // parent distance of every preorder entry = root distance of its parent
        // (recovered as the smallest root distance among ancestors: the parent of
        // entry w is the last earlier entry with a smaller distance on its root path)
        const size_t end = vtx.size();
        std::vector<int32_t> anc;
        for (size_t i = start; i < end; ++i) {
            // ancestors of vtx[i] on the preorder stack: pop entries that are not ancestors
            const int32_t v = vtx[i];
            while (!anc.empty()) {
                const int32_t a = anc.back();
                bool is_parent = false;
                for (int64_t e = hp.ptr[size_t(v)]; e < hp.ptr[size_t(v) + 1]; ++e)
                    if (hp.adj[size_t(e)] == a && dd[size_t(a)] < dd[size_t(v)]) is_parent = true;
                if (is_parent) break;
                anc.pop_back();
            }
            pdist.push_back(anc.empty() ? 0 : int32_t(dd[size_t(anc.back())]));
            anc.push_back(v);
        }
        // exact diameter: farthest from the root, then farthest from that vertex
        int32_t far = vtx[start];
        for (size_t i = start; i < end; ++i)
            if (dd[size_t(vtx[i])] > dd[size_t(far)]) far = vtx[i];
        {
            std::vector<int64_t> d2;
            std::vector<int32_t> q(1, far);
            std::vector<char> s2;
            std::map<int32_t, int64_t> dmap;
            dmap[far] = 0;
            for (size_t h = 0; h < q.size(); ++h) {
                const int32_t a = q[h];
                for (int64_t e = hp.ptr[size_t(a)]; e < hp.ptr[size_t(a) + 1]; ++e) {
                    const int32_t b = hp.adj[size_t(e)];
                    if (dmap.count(b)) continue;
                    dmap[b] = dmap[a] + hp.qlen[size_t(e)];
                    max_diam = std::max(max_diam, dmap[b]);
                    q.push_back(b);
                }
            }
        }
        tree_ptr.push_back(int32_t(end));
        max_tree = std::max<int32_t>(max_tree, int32_t(end - start));
    }
    if (max_diam >= tfi::kGridMax) return fail(TFI_ERR_GRID_OVERFLOW, "tree diameter beyond 2^30 grid units");
    if (hp.f.kind == TFI_F_TABLE && max_diam >= int64_t(hp.f.table.size()))
        return fail(TFI_ERR_GRID_OVERFLOW, "sampled kernel table shorter than the largest tree diameter");
    std::vector<float> ftab(size_t(max_diam + 1));
    for (int64_t k = 0; k <= max_diam; ++k) ftab[size_t(k)] = float(hp.f.grid(k, hp.delta));
    int levels = 1;
    while ((2 << (levels - 1)) <= max_tree) ++levels;
    if (tfi_status rc = p->upload(&p->dn_tree_ptr, tree_ptr)) return rc;
    if (tfi_status rc = p->upload(&p->dn_vtx, vtx)) return rc;
    if (tfi_status rc = p->upload(&p->dn_dist, dist)) return rc;
    if (tfi_status rc = p->upload(&p->dn_ftab, ftab)) return rc;
    p->dense_ftab_len = int64_t(ftab.size());
    void *st = nullptr, *errp = nullptr;
    if (tfi_status rc = p->alloc(&st, size_t(levels) * size_t(n) * 4)) return rc;
    if (tfi_status rc = p->alloc(&errp, 16)) return rc;
    p->dn_st = static_cast<int32_t *>(st);
    p->dn_err = static_cast<int32_t *>(errp);
    TFI_CUDA(cudaMemset(p->dn_err, 0, 16));
    TFI_CUDA(cudaMemcpy(p->dn_st, pdist.data(), size_t(n) * 4, cudaMemcpyHostToDevice));
    for (int l = 1; l < levels; ++l)
        tfi::tc::sparse_level<<<grid_for(n, 256), 256>>>(p->dn_st + int64_t(l - 1) * n, p->dn_st + int64_t(l) * n, n,
                                                         1 << (l - 1));
    TFI_CUDA(cudaGetLastError());
    TFI_CUDA(cudaDeviceSynchronize());
    p->dense_trees = int32_t(tree_ptr.size()) - 1;
    p->dense_levels = levels;
    p->dense_max_tree = max_tree;
    p->dn_tree_ptr_h = tree_ptr;
    p->dense_ready = true;
    return TFI_OK;
}

template <typename T, int NC>
tfi_status dense_impl(tfi_plan_t p, const T *F, T *out, int d, cudaStream_t s) {
    if (tfi_status rc = build_dense(p)) return rc;
    constexpr size_t smem = tfi::tc::dense_smem_bytes<T, NC>();
    TFI_CUDA(cudaFuncSetAttribute(tfi::tc::dense_tc_kernel<T, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(smem)));
    std::vector<tfi::tc::DenseItem> items;
    for (int t = 0; t < p->dense_trees; ++t)
        for (int32_t t0 = p->dn_tree_ptr_h[size_t(t)]; t0 < p->dn_tree_ptr_h[size_t(t) + 1]; t0 += tfi::tc::kTileM)
            for (int c0 = 0; c0 < d; c0 += NC) items.push_back(tfi::tc::DenseItem{t0, t, c0, 0});
    tfi::tc::DenseItem *d_items = nullptr;
    TFI_CUDA(cudaMalloc(&d_items, items.size() * sizeof(items[0])));
    TFI_CUDA(cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(items[0]), cudaMemcpyHostToDevice, s));
    tfi::tc::dense_tc_kernel<T, NC><<<unsigned(items.size()), 128, smem, s>>>(
        d_items, p->dn_tree_ptr, p->dn_vtx, p->dn_dist, p->dn_st, int64_t(p->hp.n), p->dense_levels, p->dn_ftab, F, d,
        out, p->dn_err);
    const cudaError_t le = cudaGetLastError();
    const cudaError_t se = cudaStreamSynchronize(s);
    cudaFree(d_items);
    if (le != cudaSuccess) return fail(TFI_ERR_CUDA, std::string("dense_tc_kernel launch: ") + cudaGetErrorString(le));
    if (se != cudaSuccess) return fail(TFI_ERR_CUDA, std::string("dense_tc_kernel: ") + cudaGetErrorString(se));
    int32_t err = 0;
    TFI_CUDA(cudaMemcpy(&err, p->dn_err, 4, cudaMemcpyDeviceToHost));
    if (err) {
        cudaMemset(p->dn_err, 0, 4);
        return fail(TFI_ERR_TIMEOUT, "a tensor-core completion wait gave up");
    }
    return TFI_OK;
}

// ---------------------------------------------------------------------------
// kernel gradient
// ---------------------------------------------------------------------------
tfi_status build_grad(tfi_plan_t p) {
    if (p->grad_ready) return TFI_OK;
    const tfi::HostPlan &hp = p->hp;
    // the gradient counts pairs at every distance: the jobs before any support truncation
    const std::vector<tfi::Job> &gjobs = hp.jobs_full.empty() ? hp.jobs : hp.jobs_full;
    std::vector<tfi::grad::GradJob> gj;
    std::vector<int64_t> seg_off;
    std::vector<int32_t> seg_len;
    std::vector<float> seg_sign;
    int64_t hoff = 0, moff = 0;
    int max_lnp = 0;
    const int nblk = (hp.max_channels + tfi::grad::kGradCB - 1) / tfi::grad::kGradCB;
    const int64_t ncb_max = (hp.max_channels + tfi::grad::kGradDotCB - 1) / tfi::grad::kGradDotCB;
    std::vector<int64_t> ditems;  // direct jobs: (job << 16 | row tile << 8 | column tile) items
    std::vector<int32_t> djobs;   // and the direct jobs' indices
    for (const tfi::Job &j : gjobs) {
        if (j.ke == j.kb) continue;
        const int32_t len = 2 * j.maxr + j.maxx + 1;
        // direct evaluation (pair dot products over the channels, then one binning pass) when it is cheaper
        // than one FFT correlation per channel at max_channels; a table beyond one shared-memory
        // transform (P1 P2 > 2^13) takes the direct evaluation whatever its size class
        const double nk = double(j.ke - j.kb), D = double(hp.max_channels);
        const double np = std::ldexp(1.0, j.lp1 + j.lp2);
        const double cost_direct = 2 * nk * nk * D + 64 * nk * nk;   // pair dot products, one binning pass
        const double cost_fft = D * (5 * np * std::max(1, j.lp1 + j.lp2) + 10 * np);
        const bool fft_ok = j.lp1 + j.lp2 <= 13, direct_ok = nk <= 32 * 255;
        if (!fft_ok && !direct_ok)
            return fail(TFI_ERR_UNSUPPORTED, "kernel gradient: a table has more than 2^13 points and more than 8160 "
                                             "occupied bins (neither evaluator of the correlation takes it)");
        const int32_t mode = (direct_ok && (!fft_ok || cost_direct < cost_fft)) ? 1 : 0;
        gj.push_back(tfi::grad::GradJob{int32_t(j.kb), int32_t(j.ke), j.lp1, j.lp2, j.maxr, j.maxx, hoff, mode, 0,
                                        mode ? moff : 0});
        if (mode) {
            const int32_t nt = int32_t((j.ke - j.kb + 31) / 32);
            for (int32_t a = 0; a < nt; ++a)
                for (int32_t b = 0; b < nt; ++b) ditems.push_back((int64_t(gj.size() - 1) << 16) | (a << 8) | b);
            djobs.push_back(int32_t(gj.size() - 1));
            p->g_dir_max_k = std::max(p->g_dir_max_k, 2 * j.maxr + j.maxx + 1);
            p->g_dir_max_nk = std::max(p->g_dir_max_nk, int32_t(j.ke - j.kb));
            moff += int64_t(j.ke - j.kb) * (j.ke - j.kb) * ncb_max;  // one partial product per channel block
        }
        seg_off.push_back(hoff);
        seg_len.push_back(len);
        seg_sign.push_back(j.is_comp ? -1.f : 1.f);
        hoff += int64_t(len) * nblk;  // one histogram per channel block; the job's sum lands in the first
        if (mode == 0) max_lnp = std::max(max_lnp, j.lp1 + j.lp2);  // sizes grad_fft_kernel's shared memory
    }
    std::vector<int32_t> leaf_ptr(1, 0), hist_len;
    std::vector<int64_t> pair_off, hist_off;
    int64_t poff = 0;
    int32_t leaf_max_n = 1, leaf_max_hl = 1;
    const int64_t leaf_hbase = hoff;
    for (const tfi::Leaf &lf : hp.leaves) {
        const int64_t sz = lf.end - lf.begin;
        leaf_max_n = std::max(leaf_max_n, int32_t(sz));
        leaf_max_hl = std::max(leaf_max_hl, int32_t(lf.diam + 1));
        leaf_ptr.push_back(int32_t(lf.end));
        pair_off.push_back(poff);
        poff += sz * sz;
        hist_off.push_back(hoff);
        hist_len.push_back(int32_t(lf.diam + 1));
        seg_off.push_back(hoff);
        seg_len.push_back(int32_t(lf.diam + 1));
        seg_sign.push_back(1.f);
        hoff += lf.diam + 1;
    }
    {
        // segments longest first (grad_reduce's prefix search), ties in their original order
        std::vector<size_t> ord(seg_len.size());
        for (size_t q = 0; q < ord.size(); ++q) ord[q] = q;
        std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return seg_len[a] > seg_len[b]; });
        std::vector<int64_t> so(ord.size());
        std::vector<int32_t> sl(ord.size());
        std::vector<float> ss(ord.size());
        for (size_t q = 0; q < ord.size(); ++q) {
            so[q] = seg_off[ord[q]];
            sl[q] = seg_len[ord[q]];
            ss[q] = seg_sign[ord[q]];
        }
        seg_off.swap(so);
        seg_len.swap(sl);
        seg_sign.swap(ss);
    }
    {
        std::vector<int32_t> f1;
        p->g_fft1d_cls.assign(16, 0);
        for (int ln = 1; ln <= 14; ++ln) {
            p->g_fft1d_cls[size_t(ln)] = int32_t(f1.size());
            for (size_t q = 0; q < gj.size(); ++q)
                if (gj[q].mode == 0 && gj[q].lp2 == 0 && gj[q].lp1 == ln) f1.push_back(int32_t(q));
        }
        p->g_fft1d_cls[15] = int32_t(f1.size());
        if (tfi_status rc = p->upload(&p->g_fft1d, f1)) return rc;
        p->n_gfft1d = int32_t(f1.size());
    }
    if (tfi_status rc = p->upload(&p->g_jobs, gj)) return rc;
    if (tfi_status rc = p->upload(&p->g_leaf_ptr, leaf_ptr)) return rc;
    if (tfi_status rc = p->upload(&p->g_pair_off, pair_off)) return rc;
    if (tfi_status rc = p->upload(&p->g_hist_off, hist_off)) return rc;
    if (tfi_status rc = p->upload(&p->g_hist_len, hist_len)) return rc;
    if (tfi_status rc = p->upload(&p->g_seg_off, seg_off)) return rc;
    if (tfi_status rc = p->upload(&p->g_seg_len, seg_len)) return rc;
    if (tfi_status rc = p->upload(&p->g_seg_sign, seg_sign)) return rc;
    void *q = nullptr;
    if (tfi_status rc = p->alloc(&q, size_t(std::max<int64_t>(hoff, 1)) * 4)) return rc;
    p->g_hist = static_cast<float *>(q);
    p->g_leaf_max_n = leaf_max_n;
    p->g_leaf_max_hl = leaf_max_hl;
    p->g_leaf_onepass = tfi::grad::grad_leaf_warp_smem(leaf_max_n, leaf_max_hl) <= size_t(227 * 1024);
    p->g_leaf_hbase = leaf_hbase;
    p->g_leaf_hlen = hoff - leaf_hbase;
    if (p->g_leaf_onepass) {
        if (tfi_status rc = p->alloc(&q, std::max<size_t>(1, hp.leaves.size()) * 4)) return rc;
        p->g_leaf_S = static_cast<int32_t *>(q);
        if (tfi_status rc = p->alloc(&q, size_t(std::max<int64_t>(p->g_leaf_hlen, 1)) * 8)) return rc;
        p->g_h64 = static_cast<unsigned long long *>(q);
    } else {
        // leaves with long histograms: pair values and distances in global memory, then binned
        if (tfi_status rc = p->alloc(&q, size_t(std::max<int64_t>(poff, 1)) * 4)) return rc;
        p->g_pval = static_cast<float *>(q);
        if (tfi_status rc = p->alloc(&q, size_t(std::max<int64_t>(poff, 1)) * 4)) return rc;
        p->g_pdst = static_cast<int32_t *>(q);
    }
    if (tfi_status rc = p->alloc(&q, std::max<size_t>(1, hp.key_r.size()) * size_t(hp.max_channels) * 4)) return rc;
    p->g_gbuf = static_cast<float *>(q);
    if (tfi_status rc = p->alloc(&q, size_t(hp.hist_len) * 8)) return rc;
    p->g_C = static_cast<double *>(q);
    if (tfi_status rc = p->alloc(&q, std::max<size_t>(1, hp.f.params.size()) * 8 * 2)) return rc;
    p->g_params = static_cast<double *>(q);
    p->g_dtheta = p->g_params + std::max<size_t>(1, hp.f.params.size());
    p->n_gjobs = int32_t(gj.size());
    p->n_gleaves = int32_t(hp.leaves.size());
    p->n_gseg = int32_t(seg_off.size());
    p->g_max_lnp = max_lnp;
    p->g_nblk = nblk;
    if (tfi_status rc = p->upload(&p->g_ditems, ditems)) return rc;
    if (tfi_status rc = p->upload(&p->g_djobs, djobs)) return rc;
    if (tfi_status rc = p->alloc(&q, size_t(std::max<int64_t>(moff, 1)) * 4)) return rc;
    p->g_M = static_cast<float *>(q);
    p->n_gditems = int32_t(ditems.size());
    p->n_gdjobs = int32_t(djobs.size());
    p->grad_ready = true;
    return TFI_OK;
}

template <typename T>
tfi_status kernel_grad_impl(tfi_plan_t p, const T *G, const T *F, int d, double *C, double *dtheta, cudaStream_t s) {
    if (tfi_status rc = build_grad(p)) return rc;
    const tfi::HostPlan &hp = p->hp;
    const int64_t n_keys = int64_t(hp.key_r.size());
    if (n_keys > 0) {
        // the bin sums of g and F, by the apply's segmented kernel (the same fixed summation order)
        launch_bucket(p, G, d, s, p->g_gbuf);
        launch_bucket(p, F, d, s, p->kbuf);
    }
    if (p->n_gjobs > 0) {
        const size_t smem = 2 * size_t(tfi::dev::padded_size(1 << p->g_max_lnp)) * sizeof(float2);
        TFI_CUDA(cudaFuncSetAttribute(tfi::grad::grad_fft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      int(std::max<size_t>(smem, 1024))));
        const int nb = (d + tfi::grad::kGradCB - 1) / tfi::grad::kGradCB;  // channel blocks with channels
        tfi::grad::grad_fft_kernel<<<dim3(unsigned(p->n_gjobs), unsigned(nb)), 256, smem, s>>>(
            p->g_jobs, p->key_r, p->key_x, d, p->g_gbuf, p->kbuf, p->twiddle, p->g_hist);
        // one launch per transform size, each with the shared memory of its size
        for (int ln = 1; ln <= 14 && p->n_gfft1d > 0; ++ln) {
            const int b0 = p->g_fft1d_cls[size_t(ln)], b1 = p->g_fft1d_cls[size_t(ln) + 1];
            if (b1 == b0) continue;
            const size_t sm1 = size_t(1 << ln) * 16 + size_t(tfi::dev::padded_size(1 << ln)) * sizeof(float2);
            TFI_CUDA(cudaFuncSetAttribute(tfi::grad::grad_fft1d_x2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          int(sm1)));
            tfi::grad::grad_fft1d_x2_kernel<<<dim3(unsigned(b1 - b0), unsigned(nb)), 256, sm1, s>>>(
                p->g_jobs, p->g_fft1d + b0, p->key_r, d, p->g_gbuf, p->kbuf, p->twiddle,
                reinterpret_cast<const ulonglong2 *>(p->twiddle_b), p->g_hist);
        }
        if (nb > 1) tfi::grad::grad_block_reduce<<<p->n_gjobs, 128, 0, s>>>(p->g_jobs, p->n_gjobs, nb, p->g_hist);
        if (p->n_gditems > 0) {
            const int ncb = (d + tfi::grad::kGradDotCB - 1) / tfi::grad::kGradDotCB;
            tfi::grad::grad_pair_dots<<<dim3(unsigned(p->n_gditems), unsigned(ncb)), 256, 0, s>>>(
                p->g_jobs, p->g_ditems, d, p->g_gbuf, p->kbuf, p->g_M);
            const size_t dsm = tfi::grad::grad_direct_bin_smem(p->g_dir_max_k, p->g_dir_max_nk);
            if (dsm <= size_t(200 * 1024)) {
                TFI_CUDA(cudaFuncSetAttribute(tfi::grad::grad_direct_bin_fx,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, int(dsm)));
                tfi::grad::grad_direct_bin_fx<<<p->n_gdjobs, 256, dsm, s>>>(p->g_jobs, p->g_djobs, ncb, p->key_r,
                                                                            p->key_x, p->g_dir_max_k, p->g_M,
                                                                            p->g_hist);
            } else
            tfi::grad::grad_direct_bin<<<p->n_gdjobs, 128, 0, s>>>(p->g_jobs, p->g_djobs, ncb, p->key_r, p->key_x,
                                                                   p->g_M, p->g_hist);
        }
    }
    if (p->n_gleaves > 0 && p->g_leaf_onepass) {
        const size_t smem = tfi::grad::grad_leaf_warp_smem(p->g_leaf_max_n, p->g_leaf_max_hl);
        TFI_CUDA(cudaFuncSetAttribute(tfi::grad::grad_leaf_warp_hist<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      int(smem)));
        tfi::grad::grad_leaf_scale<T><<<p->n_gleaves, 256, 0, s>>>(p->g_leaf_ptr, p->leaf_vtx, G, F, d, p->g_leaf_S);
        // few leaves with many channels: their channel blocks spread over CTAs, whose exact integer
        // sums are merged in global memory
        const int nblk = (d + 15) / 16;
        const int groups = std::max(1, std::min(nblk, (2 * device_sms() + p->n_gleaves - 1) / p->n_gleaves));
        if (groups > 1) TFI_CUDA(cudaMemsetAsync(p->g_h64, 0, size_t(p->g_leaf_hlen) * 8, s));
        tfi::grad::grad_leaf_warp_hist<T><<<dim3(unsigned(p->n_gleaves), unsigned(groups)),
                                            32 * tfi::grad::kGradLeafWarps, smem, s>>>(
            p->g_leaf_ptr, p->g_hist_off, p->g_hist_len, p->leaf_vtx, p->leaf_dist, p->leaf_pdist, G, F, d,
            p->g_leaf_max_n, p->g_leaf_max_hl, p->g_leaf_S, p->g_h64, p->g_leaf_hbase, p->g_hist);
        if (groups > 1)
            tfi::grad::grad_leaf_h64_to_float<<<p->n_gleaves, 256, 0, s>>>(p->g_leaf_S, p->g_hist_off, p->g_hist_len,
                                                                           p->g_h64, p->g_leaf_hbase, p->g_hist);
    } else if (p->n_gleaves > 0) {
        tfi::grad::grad_leaf_pairs<T><<<p->n_gleaves, 256, 0, s>>>(p->g_leaf_ptr, p->g_pair_off, p->leaf_vtx,
                                                                    p->leaf_dist, p->leaf_pdist, G, F, d, p->g_pval,
                                                                    p->g_pdst);
        tfi::grad::grad_leaf_hist<<<p->n_gleaves, 128, 0, s>>>(p->g_leaf_ptr, p->g_pair_off, p->g_hist_off,
                                                               p->g_hist_len, p->g_pval, p->g_pdst, p->g_hist);
    }
    double *Cd = C ? C : p->g_C;
    tfi::grad::grad_reduce<<<grid_for(hp.hist_len * 32, 256), 256, 0, s>>>(p->n_gseg, p->g_seg_off, p->g_seg_len,
                                                                            p->g_seg_sign, p->g_hist, hp.hist_len, Cd);
    TFI_CUDA(cudaGetLastError());
    if (dtheta && hp.f.kind != TFI_F_TABLE && !hp.f.params.empty()) {
        const int np = int(hp.f.params.size());
        // dtheta in device memory: written on the stream, no synchronisation
        cudaPointerAttributes attr{};
        const bool on_dev = cudaPointerGetAttributes(&attr, dtheta) == cudaSuccess &&
                            (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
        cudaGetLastError();  // a plain host pointer may leave an error from the query
        TFI_CUDA(cudaMemcpyAsync(p->g_params, hp.f.params.data(), size_t(np) * 8, cudaMemcpyHostToDevice, s));
        tfi::grad::grad_params<<<np, 256, 0, s>>>(hp.f.kind, p->g_params, np, hp.delta, Cd, hp.hist_len,
                                                  on_dev ? dtheta : p->g_dtheta);
        TFI_CUDA(cudaGetLastError());
        if (!on_dev) {
            TFI_CUDA(cudaMemcpyAsync(dtheta, p->g_dtheta, size_t(np) * 8, cudaMemcpyDeviceToHost, s));
            TFI_CUDA(cudaStreamSynchronize(s));
        }
    }
    return TFI_OK;
}

}  // namespace

extern "C" {

const char *tfi_last_error(void) { return g_err.c_str(); }

tfi_status tfi_plan(const tfi_tree *tree, const tfi_kernel *kernel, const tfi_options *opt, tfi_plan_t *out) {
    g_err.clear();
    if (!tree || !kernel || !opt || !out) return fail(TFI_ERR_ARG, "null argument");
    *out = nullptr;
    if (tree->n < 1 || tree->n_edges < 0 || tree->n_edges > tree->n - 1)
        return fail(TFI_ERR_ARG, "need n >= 1 and 0 <= n_edges <= n - 1");
    if (tree->n_edges > 0 && (!tree->u || !tree->v || !tree->w)) return fail(TFI_ERR_ARG, "null edge array");
    if (!(opt->delta > 0.0) || !std::isfinite(opt->delta)) return fail(TFI_ERR_ARG, "delta must be finite and > 0");
    if (opt->policy < 0 || opt->policy > 2) return fail(TFI_ERR_ARG, "unknown policy");
    if (opt->leaf_max < 1 || opt->leaf_max > tfi::kLeafMax)
        return fail(TFI_ERR_ARG, "leaf_max must be in [1, " + std::to_string(tfi::kLeafMax) + "]");
    if (opt->max_channels < 1) return fail(TFI_ERR_ARG, "max_channels must be >= 1");
    if (opt->fft_cta_points != 0 && opt->fft_cta_points != 4096 && opt->fft_cta_points != 8192 &&
        opt->fft_cta_points != 16384)
        return fail(TFI_ERR_ARG, "fft_cta_points must be 0, 4096, 8192 or 16384");
    if (kernel->kind < 0 || kernel->kind > 4) return fail(TFI_ERR_ARG, "unknown kernel kind");
    if (kernel->n_params < 0 || (kernel->n_params > 0 && !kernel->params)) return fail(TFI_ERR_ARG, "bad kernel params");
    const int need[5] = {0, 2, 2, 4, 3};
    if (kernel->kind == TFI_F_EXPSUM ? (kernel->n_params < 2 || kernel->n_params % 2)
                                     : kernel->n_params != need[kernel->kind])
        return fail(TFI_ERR_ARG, "wrong number of kernel parameters");
    if (kernel->kind == TFI_F_TABLE && (kernel->table_len < 1 || !kernel->table))
        return fail(TFI_ERR_ARG, "sampled kernel needs a table");
    std::unique_ptr<tfi_plan_s> p(new (std::nothrow) tfi_plan_s());
    if (!p) return fail(TFI_ERR_OOM, "host allocation failed");
    tfi::HostPlan &hp = p->hp;
    hp.delta = opt->delta;
    hp.policy = opt->policy;
    hp.leaf_max = opt->leaf_max;
    hp.max_channels = opt->max_channels;
    hp.flags = opt->flags;
    p->fft_cta_points = opt->fft_cta_points ? opt->fft_cta_points : kFftSmemPairPoints;
    if ((opt->flags & TFI_PLAN_SWEEP) && kernel->kind != TFI_F_EXPSUM)
        return fail(TFI_ERR_ARG, "TFI_PLAN_SWEEP needs an exponential-sum kernel (TFI_F_EXPSUM)");
    hp.f.kind = kernel->kind;
    hp.f.params.assign(kernel->params, kernel->params + kernel->n_params);
    if (kernel->kind == TFI_F_TABLE) hp.f.table.assign(kernel->table, kernel->table + kernel->table_len);
    std::string err;
    int rc;
    try {
        rc = tfi::build_plan(hp, tree->n, tree->n_edges, tree->u, tree->v, tree->w, err);
    } catch (const std::bad_alloc &) {
        return fail(TFI_ERR_OOM, "host allocation failed while planning");
    }
    if (rc) return fail(rc, err);
    if (!(opt->flags & TFI_PLAN_HOST_ONLY)) {
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
            return fail(TFI_ERR_NO_DEVICE, "no CUDA device (build with TFI_PLAN_HOST_ONLY to plan on the host)");
        if (tfi_status r2 = upload_plan(p.get())) return r2;
    }
    *out = p.release();
    return TFI_OK;
}

}  // extern "C"

namespace {

// Drop the per-d work lists (they depend on fft_cta_points); rebuilt on the next apply.
void clear_work(tfi_plan_t p) {
    for (auto &kv : p->work) {
        cudaFree(kv.second.d_fft);
        cudaFree(kv.second.d_dir);
        cudaFree(kv.second.d_tab);
        cudaFree(kv.second.d_tab_ptr);
        cudaFree(kv.second.d_hk);
        cudaFree(kv.second.d_big);
    }
    p->work.clear();
}

__global__ void fill_ones_bf16(int64_t n, __nv_bfloat16 *x) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        x[i] = __float2bfloat16_rn(1.f);
}

// The first `count` trees of a forest (ordered by their smallest vertex), relabelled in
// ascending vertex order; every tree when count <= 0 or the forest has fewer trees.
struct SubForest {
    std::vector<int32_t> u, v;
    std::vector<double> w;
    int32_t n = 0;
    bool whole = true;
};
SubForest first_trees(const tfi_tree *t, int32_t count) {
    SubForest sf;
    std::vector<int32_t> par(size_t(t->n));
    std::iota(par.begin(), par.end(), 0);
    auto find = [&](int32_t a) {
        while (par[size_t(a)] != a) a = par[size_t(a)] = par[size_t(par[size_t(a)])];
        return a;
    };
    for (int32_t e = 0; e < t->n_edges; ++e) {
        const int32_t a = find(t->u[e]), b = find(t->v[e]);
        if (a != b) par[size_t(std::max(a, b))] = std::min(a, b);  // root = smallest vertex of the tree
    }
    std::vector<int32_t> label(size_t(t->n), -1);
    int32_t trees = 0;
    for (int32_t x = 0; x < t->n; ++x) {
        const int32_t r = find(x);
        if (r == x) ++trees;
        if (count <= 0 || trees <= count) label[size_t(x)] = sf.n++;
    }
    sf.whole = count <= 0 || trees <= count;
    for (int32_t e = 0; e < t->n_edges; ++e) {
        if (label[size_t(t->u[e])] < 0) continue;
        sf.u.push_back(label[size_t(t->u[e])]);
        sf.v.push_back(label[size_t(t->v[e])]);
        sf.w.push_back(t->w[e]);
    }
    return sf;
}

}  // namespace

extern "C" {

tfi_status tfi_autotune(const tfi_tree *tree, const tfi_kernel *kernel, const tfi_options *opt, int32_t d,
                        int32_t dtype, const int32_t *leaf_candidates, int32_t n_leaf, int32_t sample_trees,
                        int32_t reps, tfi_options *tuned, double *best_ms, tfi_plan_t *plan_out) {
    if (!tree || !kernel || !opt || !tuned) return fail(TFI_ERR_ARG, "null argument");
    if (plan_out) *plan_out = nullptr;
    if (opt->flags & TFI_PLAN_HOST_ONLY) return fail(TFI_ERR_ARG, "autotuning measures on the device (no HOST_ONLY)");
    if (d < 1 || d > opt->max_channels) return fail(TFI_ERR_ARG, "d must be in [1, max_channels]");
    if (dtype != TFI_DTYPE_F32 && dtype != TFI_DTYPE_BF16) return fail(TFI_ERR_ARG, "unknown dtype");
    if (n_leaf < 0 || (n_leaf > 0 && !leaf_candidates)) return fail(TFI_ERR_ARG, "bad leaf candidates");
    if (reps < 1) return fail(TFI_ERR_ARG, "reps must be >= 1");
    if (tree->n < 1 || tree->n_edges < 0 || tree->n_edges > tree->n - 1 ||
        (tree->n_edges > 0 && (!tree->u || !tree->v || !tree->w)))
        return fail(TFI_ERR_ARG, "bad tree");
    for (int32_t e = 0; e < tree->n_edges; ++e)
        if (tree->u[e] < 0 || tree->u[e] >= tree->n || tree->v[e] < 0 || tree->v[e] >= tree->n)
            return fail(TFI_ERR_NOT_TREE, "edge endpoint out of range");
    std::vector<int32_t> cand;
    if (n_leaf > 0) cand.assign(leaf_candidates, leaf_candidates + n_leaf);
    else cand = {64, 128, 256, 512, 1024};
    const int32_t ctas[3] = {4096, 8192, 16384};
    const SubForest sf = first_trees(tree, sample_trees);
    const tfi_tree sub{sf.n, int32_t(sf.u.size()), sf.u.data(), sf.v.data(), sf.w.data()};
    const tfi_tree *tune_tree = sf.whole ? tree : &sub;
    const size_t esz = dtype == TFI_DTYPE_BF16 ? 2 : 4;
    const int64_t nd = int64_t(tune_tree->n) * d;
    struct Buffers {
        void *F = nullptr, *out = nullptr;
        cudaStream_t s = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        ~Buffers() {
            cudaFree(F);
            cudaFree(out);
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
            if (s) cudaStreamDestroy(s);
        }
    } b;
    if (cudaMalloc(&b.F, size_t(nd) * esz) != cudaSuccess || cudaMalloc(&b.out, size_t(nd) * esz) != cudaSuccess)
        return fail(TFI_ERR_OOM, "cudaMalloc failed for the autotuning fields");
    TFI_CUDA(cudaStreamCreateWithFlags(&b.s, cudaStreamNonBlocking));
    TFI_CUDA(cudaEventCreate(&b.e0));
    TFI_CUDA(cudaEventCreate(&b.e1));
    if (dtype == TFI_DTYPE_F32)
        tfi::dev::fill_value<<<grid_for(nd, 256), 256, 0, b.s>>>(nd, 1.f, static_cast<float *>(b.F));
    else
        fill_ones_bf16<<<grid_for(nd, 256), 256, 0, b.s>>>(nd, static_cast<__nv_bfloat16 *>(b.F));
    TFI_CUDA(cudaGetLastError());
    double best = INFINITY;
    tfi_options best_opt = *opt;
    tfi_plan_t keep = nullptr;
    for (int32_t s0 : cand) {
        tfi_options o = *opt;
        o.leaf_max = std::max(1, std::min(s0, tfi::kLeafMax));
        o.fft_cta_points = 0;
        tfi_plan_t pl = nullptr;
        if (tfi_status rc = tfi_plan(tune_tree, kernel, &o, &pl)) {
            tfi_destroy(keep);
            return rc;
        }
        bool kept = false;
        for (int32_t cta : ctas) {
            clear_work(pl);
            pl->fft_cta_points = cta;
            tfi_status rc = TFI_OK;
            for (int w = 0; w < 2 && rc == TFI_OK; ++w) rc = tfi_apply(pl, b.F, b.out, d, dtype, b.s);
            if (rc == TFI_OK) rc = cudaEventRecord(b.e0, b.s) == cudaSuccess ? TFI_OK : TFI_ERR_CUDA;
            for (int r = 0; r < reps && rc == TFI_OK; ++r) rc = tfi_apply(pl, b.F, b.out, d, dtype, b.s);
            float ms = 0.f;
            if (rc == TFI_OK && (cudaEventRecord(b.e1, b.s) != cudaSuccess || cudaEventSynchronize(b.e1) != cudaSuccess ||
                                 cudaEventElapsedTime(&ms, b.e0, b.e1) != cudaSuccess))
                rc = fail(TFI_ERR_CUDA, "autotuning timing failed");
            if (rc != TFI_OK) {
                tfi_destroy(pl);
                if (keep != pl) tfi_destroy(keep);
                return rc;
            }
            const double per = double(ms) / reps;
            if (per < best) {
                best = per;
                best_opt = o;
                best_opt.fft_cta_points = cta;
                if (keep && keep != pl) tfi_destroy(keep);
                keep = pl;
                kept = true;
            }
        }
        if (!kept) tfi_destroy(pl);
    }
    *tuned = best_opt;
    if (best_ms) *best_ms = best;
    if (!plan_out) {
        tfi_destroy(keep);
        return TFI_OK;
    }
    if (sf.whole) {
        // the winner's plan, with its work lists rebuilt for the chosen tile on the next apply
        clear_work(keep);
        keep->fft_cta_points = best_opt.fft_cta_points;
        *plan_out = keep;
        return TFI_OK;
    }
    tfi_destroy(keep);
    return tfi_plan(tree, kernel, &best_opt, plan_out);
}

tfi_status tfi_apply(tfi_plan_t plan, const void *F, void *out, int32_t d, int32_t dtype, tfi_stream_t stream) {
    if (tfi_status rc = check_apply_args(plan, F, out, d, dtype)) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dtype == TFI_DTYPE_F32)
        return apply_impl<float>(plan, static_cast<const float *>(F), static_cast<float *>(out), d, s);
    return apply_impl<__nv_bfloat16>(plan, static_cast<const __nv_bfloat16 *>(F), static_cast<__nv_bfloat16 *>(out),
                                     d, s);
}

tfi_status tfi_apply_backward(tfi_plan_t plan, const void *grad_out, void *grad_F, int32_t d, int32_t dtype,
                              tfi_stream_t stream) {
    // K is symmetric: the adjoint is the same integrator applied to grad_out
    return tfi_apply(plan, grad_out, grad_F, d, dtype, stream);
}

tfi_status tfi_dense_apply(tfi_plan_t plan, const void *F, void *out, int32_t d, int32_t dtype,
                           tfi_stream_t stream) {
    if (tfi_status rc = check_apply_args(plan, F, out, d, dtype)) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dtype == TFI_DTYPE_F32)
        return dense_impl<float, 16>(plan, static_cast<const float *>(F), static_cast<float *>(out), d, s);
    return dense_impl<__nv_bfloat16, 64>(plan, static_cast<const __nv_bfloat16 *>(F),
                                         static_cast<__nv_bfloat16 *>(out), d, s);
}

tfi_status tfi_apply_static(tfi_plan_t plan, const void *F, void *out, int32_t d, int32_t dtype,
                            tfi_stream_t stream) {
    if (tfi_status rc = check_apply_args(plan, F, out, d, dtype)) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dtype == TFI_DTYPE_F32)
        return apply_static_impl<float>(plan, static_cast<const float *>(F), static_cast<float *>(out), d, s);
    return apply_static_impl<__nv_bfloat16>(plan, static_cast<const __nv_bfloat16 *>(F),
                                            static_cast<__nv_bfloat16 *>(out), d, s);
}

tfi_status tfi_apply_host(tfi_plan_t plan, const void *F_host, void *out_host, int32_t d, int32_t dtype,
                          tfi_stream_t stream) {
    if (!plan || !F_host || !out_host) return fail(TFI_ERR_ARG, "null argument");
    if (!plan->on_device) return fail(TFI_ERR_NO_DEVICE, "plan was built host-only");
    const size_t esz = dtype == TFI_DTYPE_BF16 ? 2 : 4;
    const size_t bytes = size_t(plan->hp.n) * size_t(d) * esz;
    if (!plan->stage_in) {
        const size_t cap = size_t(plan->hp.n) * size_t(plan->hp.max_channels) * 4;
        if (tfi_status rc = plan->alloc(&plan->stage_in, cap)) return rc;
        if (tfi_status rc = plan->alloc(&plan->stage_out, cap)) return rc;
    }
    if (tfi_status rc = check_apply_args(plan, plan->stage_in, plan->stage_out, d, dtype)) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    TFI_CUDA(cudaMemcpyAsync(plan->stage_in, F_host, bytes, cudaMemcpyHostToDevice, s));
    if (tfi_status rc = tfi_apply(plan, plan->stage_in, plan->stage_out, d, dtype, stream)) return rc;
    TFI_CUDA(cudaMemcpyAsync(out_host, plan->stage_out, bytes, cudaMemcpyDeviceToHost, s));
    TFI_CUDA(cudaStreamSynchronize(s));
    return TFI_OK;
}

tfi_status tfi_apply_host_many(tfi_plan_t plan, int32_t n_fields, const void *const *F_host, void *const *out_host,
                               int32_t d, int32_t dtype, tfi_stream_t stream) {
    if (!plan || n_fields < 0 || (n_fields > 0 && (!F_host || !out_host))) return fail(TFI_ERR_ARG, "null argument");
    if (!plan->on_device) return fail(TFI_ERR_NO_DEVICE, "plan was built host-only");
    for (int32_t i = 0; i < n_fields; ++i)
        if (!F_host[i] || !out_host[i]) return fail(TFI_ERR_ARG, "null field pointer");
    if (n_fields == 0) return TFI_OK;
    if (!plan->pipe_in[0]) {
        const size_t cap = size_t(plan->hp.n) * size_t(plan->hp.max_channels) * 4;
        for (int k = 0; k < 2; ++k) {
            if (tfi_status rc = plan->alloc(&plan->pipe_in[k], cap)) return rc;
            if (tfi_status rc = plan->alloc(&plan->pipe_out[k], cap)) return rc;
        }
        TFI_CUDA(cudaStreamCreateWithFlags(&plan->pipe_cin, cudaStreamNonBlocking));
        TFI_CUDA(cudaStreamCreateWithFlags(&plan->pipe_cout, cudaStreamNonBlocking));
        for (cudaEvent_t *e : {&plan->ev_in_ready[0], &plan->ev_in_ready[1], &plan->ev_in_free[0], &plan->ev_in_free[1],
                               &plan->ev_out_ready[0], &plan->ev_out_ready[1], &plan->ev_out_free[0],
                               &plan->ev_out_free[1]})
            TFI_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    }
    if (tfi_status rc = check_apply_args(plan, plan->pipe_in[0], plan->pipe_out[0], d, dtype)) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t bytes = size_t(plan->hp.n) * size_t(d) * (dtype == TFI_DTYPE_BF16 ? 2 : 4);
    // the copy streams start after the work already queued on the caller's stream
    TFI_CUDA(cudaEventRecord(plan->ev_fork, s));
    TFI_CUDA(cudaStreamWaitEvent(plan->pipe_cin, plan->ev_fork, 0));
    TFI_CUDA(cudaStreamWaitEvent(plan->pipe_cout, plan->ev_fork, 0));
    for (int32_t i = 0; i < n_fields; ++i) {
        const int k = i & 1;
        // copy-in: slot k's input is free once the apply of field i - 2 has read it
        if (i >= 2) TFI_CUDA(cudaStreamWaitEvent(plan->pipe_cin, plan->ev_in_free[k], 0));
        TFI_CUDA(cudaMemcpyAsync(plan->pipe_in[k], F_host[i], bytes, cudaMemcpyHostToDevice, plan->pipe_cin));
        TFI_CUDA(cudaEventRecord(plan->ev_in_ready[k], plan->pipe_cin));
        // apply on the caller's stream once the input has arrived and slot k's output of field i - 2
        // has been copied out
        TFI_CUDA(cudaStreamWaitEvent(s, plan->ev_in_ready[k], 0));
        if (i >= 2) TFI_CUDA(cudaStreamWaitEvent(s, plan->ev_out_free[k], 0));
        if (tfi_status rc = tfi_apply(plan, plan->pipe_in[k], plan->pipe_out[k], d, dtype, stream)) return rc;
        TFI_CUDA(cudaEventRecord(plan->ev_in_free[k], s));
        TFI_CUDA(cudaEventRecord(plan->ev_out_ready[k], s));
        // copy-out
        TFI_CUDA(cudaStreamWaitEvent(plan->pipe_cout, plan->ev_out_ready[k], 0));
        TFI_CUDA(cudaMemcpyAsync(out_host[i], plan->pipe_out[k], bytes, cudaMemcpyDeviceToHost, plan->pipe_cout));
        TFI_CUDA(cudaEventRecord(plan->ev_out_free[k], plan->pipe_cout));
    }
    TFI_CUDA(cudaStreamSynchronize(plan->pipe_cout));
    TFI_CUDA(cudaStreamSynchronize(plan->pipe_cin));
    TFI_CUDA(cudaStreamSynchronize(s));
    return TFI_OK;
}

}  // extern "C"

struct tfi_graph_s {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ~tfi_graph_s() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    }
};

extern "C" {

tfi_status tfi_graph_create(tfi_plan_t plan, const void *F, void *out, const void *grad_out, void *grad_F, int32_t d,
                            int32_t dtype, tfi_stream_t stream, tfi_graph_t *graph) {
    if (!graph) return fail(TFI_ERR_ARG, "null graph handle");
    *graph = nullptr;
    if (tfi_status rc = check_apply_args(plan, F, out, d, dtype)) return rc;
    const bool bwd = grad_out && grad_F;
    if (bwd) {
        if (tfi_status rc = check_apply_args(plan, grad_out, grad_F, d, dtype)) return rc;
    }
    // everything that allocates or sets attributes happens before capture
    WorkLists *wl = nullptr;
    if (tfi_status rc = build_work(plan, d, &wl)) return rc;
    if (tfi_status rc = set_attributes()) return rc;
    // capture on a private stream (the legacy default stream cannot be captured);
    // the instantiated graph may then be launched on any stream
    (void)stream;
    std::unique_ptr<tfi_graph_s> g(new (std::nothrow) tfi_graph_s());
    if (!g) return fail(TFI_ERR_OOM, "host allocation failed");
    cudaStream_t s = nullptr;
    TFI_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamDestroy(s); }
    } guard{s};
    TFI_CUDA(cudaDeviceSynchronize());
    TFI_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    tfi_status rc = tfi_apply(plan, F, out, d, dtype, s);
    if (rc == TFI_OK && bwd) rc = tfi_apply_backward(plan, grad_out, grad_F, d, dtype, s);
    cudaGraph_t gr = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(s, &gr);
    if (rc != TFI_OK) {
        if (gr) cudaGraphDestroy(gr);
        return rc;
    }
    if (ce != cudaSuccess) return fail(TFI_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ce));
    g->graph = gr;
    TFI_CUDA(cudaGraphInstantiate(&g->exec, gr, 0));
    *graph = g.release();
    return TFI_OK;
}

tfi_status tfi_sinkhorn(tfi_plan_t plan, const float *a, const float *b, float *u, float *v, int32_t d, int32_t iters,
                        double delta_reg, tfi_stream_t stream) {
    if (!plan || !a || !b || !u || !v) return fail(TFI_ERR_ARG, "null argument");
    if (iters < 0 || !(delta_reg >= 0.0)) return fail(TFI_ERR_ARG, "need iters >= 0 and delta_reg >= 0");
    if (tfi_status rc = check_apply_args(plan, u, v, d, TFI_DTYPE_F32)) return rc;
    const int64_t nd = int64_t(plan->hp.n) * d;
    if (!plan->sk_buf) {
        void *q = nullptr;
        if (tfi_status rc = plan->alloc(&q, size_t(plan->hp.n) * size_t(plan->hp.max_channels) * 4)) return rc;
        plan->sk_buf = static_cast<float *>(q);
    }
    WorkLists *wl = nullptr;
    if (tfi_status rc = build_work(plan, d, &wl)) return rc;
    if (tfi_status rc = set_attributes()) return rc;
    cudaStream_t us = static_cast<cudaStream_t>(stream);
    // u0 = v0 = 1
    tfi::dev::fill_value<<<grid_for(nd, 256), 256, 0, us>>>(nd, 1.f, u);
    tfi::dev::fill_value<<<grid_for(nd, 256), 256, 0, us>>>(nd, 1.f, v);
    TFI_CUDA(cudaGetLastError());
    if (iters == 0) return TFI_OK;
    // one iteration (two applies, two scalings) captured once, replayed `iters` times
    cudaStream_t s = nullptr;
    TFI_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    struct Guard {
        cudaStream_t s;
        cudaGraph_t g = nullptr;
        cudaGraphExec_t e = nullptr;
        ~Guard() {
            if (e) cudaGraphExecDestroy(e);
            if (g) cudaGraphDestroy(g);
            cudaStreamDestroy(s);
        }
    } gd{s};
    TFI_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const float dl = float(delta_reg);
    tfi_status rc = tfi_apply(plan, v, plan->sk_buf, d, TFI_DTYPE_F32, s);
    if (rc == TFI_OK) tfi::dev::sinkhorn_scale<<<grid_for(nd, 256), 256, 0, s>>>(nd, a, plan->sk_buf, dl, u);
    if (rc == TFI_OK) rc = tfi_apply(plan, u, plan->sk_buf, d, TFI_DTYPE_F32, s);
    if (rc == TFI_OK) tfi::dev::sinkhorn_scale<<<grid_for(nd, 256), 256, 0, s>>>(nd, b, plan->sk_buf, dl, v);
    const cudaError_t ce = cudaStreamEndCapture(s, &gd.g);
    if (rc != TFI_OK) return rc;
    if (ce != cudaSuccess) return fail(TFI_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ce));
    TFI_CUDA(cudaGraphInstantiate(&gd.e, gd.g, 0));
    for (int32_t it = 0; it < iters; ++it) TFI_CUDA(cudaGraphLaunch(gd.e, us));
    TFI_CUDA(cudaStreamSynchronize(us));
    return TFI_OK;
}

tfi_status tfi_kernel_grad(tfi_plan_t plan, const void *grad_out, const void *F, int32_t d, int32_t dtype, double *C,
                           int64_t C_len, double *dtheta, tfi_stream_t stream) {
    if (!grad_out || !F) return fail(TFI_ERR_ARG, "null field pointer");
    if (tfi_status rc = check_apply_args(plan, grad_out, F, d, dtype)) return rc;
    if (C && C_len < plan->hp.hist_len) return fail(TFI_ERR_ARG, "C_len shorter than tfi_plan_info.hist_len");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dtype == TFI_DTYPE_F32)
        return kernel_grad_impl<float>(plan, static_cast<const float *>(grad_out), static_cast<const float *>(F), d, C,
                                       dtheta, s);
    return kernel_grad_impl<__nv_bfloat16>(plan, static_cast<const __nv_bfloat16 *>(grad_out),
                                           static_cast<const __nv_bfloat16 *>(F), d, C, dtheta, s);
}

tfi_status tfi_set_kernel(tfi_plan_t plan, const tfi_kernel *kernel) {
    if (!plan || !kernel) return fail(TFI_ERR_ARG, "null argument");
    tfi::HostPlan &hp = plan->hp;
    if (kernel->kind != hp.f.kind) return fail(TFI_ERR_ARG, "kernel kind differs from the plan's");
    if (kernel->kind == TFI_F_TABLE) {
        if (!kernel->table || kernel->table_len < hp.hist_len) return fail(TFI_ERR_ARG, "table too short");
    } else if (kernel->n_params != int32_t(hp.f.params.size()) || !kernel->params) {
        return fail(TFI_ERR_ARG, "number of kernel parameters differs from the plan's");
    }
    tfi::KernelFn old = hp.f;
    hp.f.params.assign(kernel->params, kernel->params + kernel->n_params);
    if (kernel->kind == TFI_F_TABLE) hp.f.table.assign(kernel->table, kernel->table + kernel->table_len);
    std::string err;
    if (int rc = tfi::sample_kernel(hp, err)) {
        hp.f = old;
        std::string e2;
        tfi::sample_kernel(hp, e2);
        return fail(rc, err);
    }
    if (plan->on_device) {
        if (!hp.ftab.empty())
            TFI_CUDA(cudaMemcpy(plan->ftab, hp.ftab.data(), hp.ftab.size() * 4, cudaMemcpyHostToDevice));
        if (!hp.spectra.empty())
            TFI_CUDA(cudaMemcpy(plan->spectra, hp.spectra.data(), hp.spectra.size() * 4, cudaMemcpyHostToDevice));
        if (!hp.sw_beta.empty()) {
            TFI_CUDA(cudaMemcpy(plan->sw_beta, hp.sw_beta.data(), hp.sw_beta.size() * 4, cudaMemcpyHostToDevice));
            TFI_CUDA(cudaMemcpy(plan->sw_coef, hp.sw_coef.data(), hp.sw_coef.size() * 4, cudaMemcpyHostToDevice));
        }
        if (plan->dense_ready) {
            // dense f samples cover the largest tree diameter
            const size_t nd = size_t(plan->dense_ftab_len);
            std::vector<float> ft(nd);
            for (size_t k = 0; k < nd; ++k) ft[k] = float(hp.f.grid(int64_t(k), hp.delta));
            TFI_CUDA(cudaMemcpy(plan->dn_ftab, ft.data(), nd * 4, cudaMemcpyHostToDevice));
        }
    }
    return TFI_OK;
}

tfi_status tfi_selftest_wait(tfi_plan_t plan, int32_t arrive, int32_t max_polls, tfi_stream_t stream) {
    if (!plan) return fail(TFI_ERR_ARG, "null plan");
    if (!plan->on_device) return fail(TFI_ERR_NO_DEVICE, "plan was built host-only");
    if (max_polls < 1 || uint32_t(max_polls) > tfi::tc::kSpinLimit)
        return fail(TFI_ERR_ARG, "max_polls must be in [1, 2^26]");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int32_t *slot = plan->hk_err + 2;  // the self-test's own error slot, counted in device_errors
    TFI_CUDA(cudaMemsetAsync(slot, 0, 4, s));
    tfi::tc::bounded_wait_probe<<<1, 32, 0, s>>>(arrive != 0, uint32_t(max_polls), slot);
    TFI_CUDA(cudaGetLastError());
    int32_t gave_up = 0;
    TFI_CUDA(cudaMemcpyAsync(&gave_up, slot, 4, cudaMemcpyDeviceToHost, s));
    TFI_CUDA(cudaStreamSynchronize(s));
    if (gave_up) return fail(TFI_ERR_TIMEOUT, "the bounded mbarrier wait gave up");
    return TFI_OK;
}

tfi_status tfi_graph_launch(tfi_graph_t graph, tfi_stream_t stream) {
    if (!graph || !graph->exec) return fail(TFI_ERR_ARG, "null graph");
    TFI_CUDA(cudaGraphLaunch(graph->exec, static_cast<cudaStream_t>(stream)));
    return TFI_OK;
}

tfi_status tfi_graph_destroy(tfi_graph_t graph) {
    delete graph;
    return TFI_OK;
}

tfi_status tfi_destroy(tfi_plan_t plan) {
    delete plan;
    return TFI_OK;
}

tfi_status tfi_plan_get_info(tfi_plan_t plan, tfi_plan_info *info) {
    if (!plan || !info) return fail(TFI_ERR_ARG, "null argument");
    const tfi::HostPlan &hp = plan->hp;
    std::memset(info, 0, sizeof(*info));
    info->n = hp.n;
    info->n_calls = int64_t(hp.calls.size());
    info->n_leaves = int64_t(hp.leaves.size());
    info->n_levels = hp.n_levels;
    info->n_records = int64_t(hp.recs.size());
    info->n_keys = int64_t(hp.key_r.size());
    for (const tfi::Job &j : hp.jobs) {
        if (j.mode == 0) {
            info->n_jobs_fft++;
            info->sum_fft_points += int64_t(1) << (j.lp1 + j.lp2);
        } else if (j.mode == 4) {
            info->n_jobs_fft_big++;
            info->sum_fft_big_points += int64_t(1) << (j.lp1 + j.lp2);
        } else if (j.mode == 1) {
            info->n_jobs_direct++;
        } else if (j.mode == 3) {
            info->n_jobs_hankel++;
        } else {
            info->n_jobs_sweep++;
        }
    }
    for (const tfi::Call &c : hp.calls) {
        info->n_centroid += c.kind;
        info->sum_table += (c.H + 1) * (c.L + 1);
    }
    for (const tfi::Leaf &l : hp.leaves) info->sum_leaf_pairs += (l.end - l.begin) * (l.end - l.begin);
    info->ftab_len = hp.ftab_len;
    info->device_bytes = plan->dev_bytes;
    info->plan_seconds = hp.plan_seconds;
    info->device_keys_ms = plan->device_keys_ms;
    info->hist_len = hp.hist_len;
    info->trunc_len = hp.trunc;
    for (size_t r = 0; r + 1 < hp.zero_ranges.size(); r += 2) info->n_zero_bins += hp.zero_ranges[r + 1] - hp.zero_ranges[r];
    if (plan->hk_err) {
        int32_t v[3] = {0, 0, 0};
        TFI_CUDA(cudaMemcpy(v, plan->hk_err, 12, cudaMemcpyDeviceToHost));
        info->device_errors += (v[0] != 0) + (v[1] != 0) + (v[2] != 0);
    }
    if (plan->dn_err) {
        int32_t v = 0;
        TFI_CUDA(cudaMemcpy(&v, plan->dn_err, 4, cudaMemcpyDeviceToHost));
        info->device_errors += v != 0;
    }
    return TFI_OK;
}

tfi_status tfi_profile_enable(tfi_plan_t plan, int32_t enable) {
    if (!plan) return fail(TFI_ERR_ARG, "null plan");
    plan->profiling = enable != 0;
    plan->serialize = enable == 2;
    plan->prof.clear();
    plan->ev_used = 0;
    return TFI_OK;
}

tfi_status tfi_profile_read(tfi_plan_t plan, double *ms, int64_t *launches) {
    if (!plan || !ms || !launches) return fail(TFI_ERR_ARG, "null argument");
    for (int i = 0; i < TFI_N_STAGES; ++i) {
        ms[i] = 0.0;
        launches[i] = 0;
    }
    for (const auto &r : plan->prof) {
        TFI_CUDA(cudaEventSynchronize(r.b));
        float t = 0.f;
        TFI_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
        ms[r.stage] += double(t);
        launches[r.stage] += r.launches;
    }
    return TFI_OK;
}

tfi_status tfi_stage_model(tfi_plan_t plan, int32_t d, int32_t dtype, double *bytes, double *flops) {
    if (!plan || !bytes || !flops || d < 1) return fail(TFI_ERR_ARG, "bad argument");
    const tfi::HostPlan &hp = plan->hp;
    const double sin = dtype == TFI_DTYPE_BF16 ? 2.0 : 4.0, D = double(d);
    for (int i = 0; i < TFI_N_STAGES; ++i) bytes[i] = flops[i] = 0.0;
    const double nleaf = double(hp.leaf_vtx.size());
    double pairs = 0;
    for (const tfi::Leaf &l : hp.leaves) pairs += double(l.end - l.begin) * double(l.end - l.begin);
    bytes[TFI_STAGE_LEAF] = nleaf * (D * sin + 5 * 4) + nleaf * D * 4;
    flops[TFI_STAGE_LEAF] = 2.0 * D * pairs;
    const double K = double(hp.key_r.size()), KV = double(hp.key_vtx.size());
    bytes[TFI_STAGE_BUCKET] = KV * (D * sin + 4) + K * 4 + K * D * 4;
    double kf = 0, kd = 0;
    for (const tfi::Job &j : hp.jobs) {
        const double nk = double(j.ke - j.kb);
        if (j.mode == 3) {
            // B = Fh A per occupied column: 2 (H + L + 1)(H + 1) flops per channel (the appendix's
            // count); each bin is read once and written twice when L > 0 (value, then + suffix)
            std::vector<uint8_t> seen(size_t(j.maxx) + 1, 0);
            double ncols = 0;
            for (int64_t k = j.kb; k < j.ke; ++k) seen[size_t(hp.key_x[size_t(k)])] = 1;
            for (uint8_t b : seen) ncols += b;
            flops[TFI_STAGE_HANKEL] += 2.0 * double(j.maxr + j.maxx + 1) * double(j.maxr + 1) * ncols * D;
            bytes[TFI_STAGE_HANKEL] += nk * ((j.maxx > 0 ? 4 : 2) * D * 4 + 8);
        } else if (j.mode == 0 || j.mode == 4) {
            const double np = std::ldexp(1.0, j.lp1 + j.lp2);
            const double lg = double(j.lp1 + j.lp2);
            kf += nk;
            // two complex transforms and one complex product per channel pair
            flops[TFI_STAGE_FFT] += std::ceil(D / 2) * (2 * 5 * np * lg + 6 * np);
            // four-step tables also pass over their padded arrays in DRAM, per channel pair: the
            // zeroed and read input half, two reads and writes of the whole, the stored output half (per plane
            // of four channels, 16 bytes a point)
            if (j.mode == 4) bytes[TFI_STAGE_FFT] += std::ceil(D / 4) * 5.5 * np * 16;
        } else if (j.mode == 2) {
            // per term: lambda^r weighting in and out, two recurrences per backbone vertex
            bytes[TFI_STAGE_SWEEP] += nk * (2 * D * 4 + 8);
            flops[TFI_STAGE_SWEEP] += double(hp.sw_beta.size()) * nk * D * 6;
        } else {
            kd += nk;
            flops[TFI_STAGE_DIRECT] += 2.0 * nk * nk * D;
        }
    }
    bytes[TFI_STAGE_FFT] += kf * (2 * D * 4 + 8);
    bytes[TFI_STAGE_DIRECT] = kd * (2 * D * 4 + 8);
    // per record two indices; per vertex its record range and leaf flag; every table row once (the
    // rows a vertex reads are shared with the other vertices of its bin); leaf rows; output rows
    const double R = double(hp.recs.size());
    bytes[TFI_STAGE_GATHER] = R * 8 + double(hp.n) * (4 + 1) + K * D * 4 + nleaf * D * 4 + double(hp.n) * D * sin;
    return TFI_OK;
}

tfi_status tfi_plan_export(tfi_plan_t plan, int32_t what, int64_t *dst, int64_t cap, int64_t *len) {
    if (!plan || !len) return fail(TFI_ERR_ARG, "null argument");
    const tfi::HostPlan &hp = plan->hp;
    std::vector<int64_t> v;
    switch (what) {
        case TFI_EXPORT_CALLS:
            for (const tfi::Call &c : hp.calls) {
                const int64_t row[7] = {c.level, c.minv, c.size, c.kind, c.bb_end - c.bb_begin, c.H, c.L};
                v.insert(v.end(), row, row + 7);
            }
            break;
        case TFI_EXPORT_BACKBONE:
            v.assign(hp.bb.begin(), hp.bb.end());
            break;
        case TFI_EXPORT_RECORDS:
            for (size_t c = 0; c < hp.calls.size(); ++c) {
                for (int64_t i = hp.calls[c].rec_begin; i < hp.calls[c].rec_end; ++i) {
                    const tfi::Rec &r = hp.recs[size_t(i)];
                    const int64_t row[5] = {int64_t(c), r.v, r.r, r.x, r.comp >= 0 ? hp.comps[size_t(r.comp)].minv : -1};
                    v.insert(v.end(), row, row + 5);
                }
            }
            break;
        case TFI_EXPORT_LEAVES:
            for (const tfi::Leaf &l : hp.leaves) {
                const int64_t row[3] = {l.level, l.minv, l.end - l.begin};
                v.insert(v.end(), row, row + 3);
            }
            break;
        case TFI_EXPORT_DEVICE_KEYS: {
            if (!plan->on_device) return fail(TFI_ERR_NO_DEVICE, "plan was built host-only");
            const size_t R = hp.recs.size();
            std::vector<int32_t> r(R), x(R);
            if (R) {
                TFI_CUDA(cudaMemcpy(r.data(), plan->dev_rec_r, R * 4, cudaMemcpyDeviceToHost));
                TFI_CUDA(cudaMemcpy(x.data(), plan->dev_rec_x, R * 4, cudaMemcpyDeviceToHost));
            }
            for (size_t c = 0; c < hp.calls.size(); ++c) {
                for (int64_t i = hp.calls[c].rec_begin; i < hp.calls[c].rec_end; ++i) {
                    const int64_t row[4] = {int64_t(c), hp.recs[size_t(i)].v, r[size_t(i)], x[size_t(i)]};
                    v.insert(v.end(), row, row + 4);
                }
            }
            break;
        }
        case TFI_EXPORT_LEAF_PACKS: {
            std::vector<int32_t> sgrp, lo, hi, bptr, blo, bhi;
            split_leaves(hp, sgrp, lo, hi);
            int32_t cap = 0;
            pack_big_leaves(lo, hi, bptr, blo, bhi, &cap);
            for (size_t b = 0; b + 1 < bptr.size(); ++b)
                for (int32_t q = bptr[b]; q < bptr[b + 1]; ++q) {
                    const int64_t row[4] = {int64_t(b), blo[size_t(q)], bhi[size_t(q)], cap};
                    v.insert(v.end(), row, row + 4);
                }
            break;
        }
        case TFI_EXPORT_LEAF_CTAS: {
            std::vector<int32_t> sgrp, lo, hi, ptr;
            split_leaves(hp, sgrp, lo, hi);
            std::vector<int2> grouped;
            int32_t max_leaf = 1;
            const int ctas = leaf32_schedule(lo, hi, 2 * device_sms(), grouped, ptr, &max_leaf);
            for (int b = 0; b < ctas; ++b)
                for (int32_t q = ptr[size_t(b)]; q < ptr[size_t(b) + 1]; ++q) {
                    const int64_t row[4] = {int64_t(b), grouped[size_t(q)].x, grouped[size_t(q)].y, ctas};
                    v.insert(v.end(), row, row + 4);
                }
            break;
        }
        case TFI_EXPORT_JOBS:
            for (const tfi::Job &j : hp.jobs) {
                const bool any = j.ke > j.kb;
                const int64_t row[7] = {j.mode, (j.mode == 0 || j.mode == 4) ? j.lp1 + j.lp2 : -1, j.is_comp, j.ke - j.kb,
                                        any ? hp.key_vtx[size_t(hp.key_ptr[size_t(j.kb)])] : -1,
                                        any ? hp.key_vtx[size_t(hp.key_ptr[size_t(j.ke)] - 1)] : -1, j.maxr};
                v.insert(v.end(), row, row + 7);
            }
            break;
        case TFI_EXPORT_GATHER_ORDER: {
            const std::vector<int32_t> order = depth_first_order(hp);
            v.assign(order.begin(), order.end());
            break;
        }
        default:
            return fail(TFI_ERR_ARG, "unknown export");
    }
    *len = int64_t(v.size());
    if (dst && cap >= int64_t(v.size())) std::memcpy(dst, v.data(), v.size() * sizeof(int64_t));
    return TFI_OK;
}

}  // extern "C"
