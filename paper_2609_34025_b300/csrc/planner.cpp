// Host-side decomposition planner (see planner.hpp).
#include "planner.hpp"

#include "hankel_layout.hpp"

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <complex>
#include <deque>
#include <numeric>
#include <thread>

#include "tfi.h"

namespace tfi {

double KernelFn::grid(int64_t k, double delta) const {
    const double x = double(k) * delta;
    switch (kind) {
        case TFI_F_TABLE:
            return k < int64_t(table.size()) ? table[size_t(k)] : NAN;
        case TFI_F_EXPSUM: {
            double s = 0.0;
            for (size_t i = 0; i + 1 < params.size(); i += 2) s += params[i] * std::exp(-params[i + 1] * x);
            return s;
        }
        case TFI_F_GAUSS:
            return params[0] * std::exp(-params[1] * x * x);
        case TFI_F_RATIONAL:
            return params[0] / std::pow(1.0 + params[1] * std::pow(x, params[2]), params[3]);
        case TFI_F_POWEXP:
            return params[0] * std::pow(x, params[1]) * std::exp(-params[2] * x);
    }
    return NAN;
}

namespace {

struct Decomp {
    std::vector<int32_t> P;        // backbone p_1..p_m
    std::vector<int64_t> X;        // grid coordinate of each p_j (X[0] = 0)
    std::vector<int32_t> cptr;     // component ranges in cv
    std::vector<int32_t> cv;       // component vertices, traversal order from the component root
    std::vector<int64_t> cd;       // depth d(u) of each cv entry
    std::vector<int32_t> canchor;  // anchor index a(alpha)
    std::vector<int64_t> cH;       // H_alpha
    int64_t H = 0;
    void clear() {
        P.clear(); X.clear(); cptr.assign(1, 0); cv.clear(); cd.clear(); canchor.clear(); cH.clear(); H = 0;
    }
};

int ceil_log2(int64_t v) {
    int l = 0;
    while ((int64_t(1) << l) < v) ++l;
    return l;
}

uint32_t bitrev(uint32_t k, int bits) {
    // byte-wise through a 256-entry table, then shifted down to `bits` bits
    static const auto tab = [] {
        std::array<uint8_t, 256> t{};
        for (int b = 0; b < 256; ++b) {
            uint8_t r = 0;
            for (int i = 0; i < 8; ++i) r = uint8_t(r | (((b >> i) & 1) << (7 - i)));
            t[size_t(b)] = r;
        }
        return t;
    }();
    if (bits == 0) return 0;
    const uint32_t r = (uint32_t(tab[k & 255]) << 24) | (uint32_t(tab[(k >> 8) & 255]) << 16) |
                       (uint32_t(tab[(k >> 16) & 255]) << 8) | uint32_t(tab[(k >> 24) & 255]);
    return r >> (32 - bits);
}

// Run fn(i) for i in [0, n) on all hardware threads (dynamic scheduling).
template <typename Fn>
void parallel_for(size_t n, Fn fn) {
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const size_t nth = std::min<size_t>(n, hw);
    std::atomic<size_t> next(0);
    auto worker = [&]() {
        for (;;) {
            const size_t i = next.fetch_add(1);
            if (i >= n) break;
            fn(i);
        }
    };
    std::vector<std::thread> pool;
    for (size_t t = 1; t < nth; ++t) pool.emplace_back(worker);
    if (n) worker();
    for (std::thread &th : pool) th.join();
}

// Forward DFT in place of 2^lg contiguous points (natural order in and out), FP64,
// radix-2 with a table of the 2^(lg-1) roots exp(-2 pi i k / 2^lg) (w).
void fft64_tab(std::complex<double> *a, int lg, const std::complex<double> *w) {
    const int64_t n = int64_t(1) << lg;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t j = bitrev(uint32_t(i), lg);
        if (i < j) std::swap(a[i], a[j]);
    }
    for (int ll = 1; ll <= lg; ++ll) {
        const int64_t len = int64_t(1) << ll, half = len >> 1, step = n >> ll;
        for (int64_t i = 0; i < n; i += len) {
            for (int64_t k = 0; k < half; ++k) {
                const std::complex<double> x = a[i + k], y = a[i + k + half] * w[k * step];
                a[i + k] = x + y;
                a[i + k + half] = x - y;
            }
        }
    }
}

std::vector<std::complex<double>> roots64(int lg) {
    const int64_t n = int64_t(1) << lg;
    std::vector<std::complex<double>> w(size_t(std::max<int64_t>(1, n / 2)));
    for (int64_t k = 0; k < n / 2; ++k) {
        const double ang = -2.0 * M_PI * double(k) / double(n);
        w[size_t(k)] = std::complex<double>(std::cos(ang), std::sin(ang));
    }
    return w;
}

// Forward DFT of 2^lg points spaced `stride` apart (natural order in and out), FP64.
// Up to 2^14 points directly; longer ones by the four-step split n = n1 n2 (DFTs of
// length n1 over strided columns, twiddles w_n^{j2 k1}, DFTs of length n2 over
// rows, then X[k1 + n1 k2] from row k1), with the columns and rows on all host
// threads when `par` is set.
void fft64_any(std::complex<double> *a, int lg, int64_t stride, bool par) {
    const int64_t n = int64_t(1) << lg;
    std::vector<std::complex<double>> t(static_cast<size_t>(n));
    for (int64_t i = 0; i < n; ++i) t[size_t(i)] = a[i * stride];
    if (lg <= 14) {
        const std::vector<std::complex<double>> w = roots64(lg);
        fft64_tab(t.data(), lg, w.data());
    } else {
        const int l1 = lg / 2, l2 = lg - l1;
        const int64_t n1 = int64_t(1) << l1, n2 = int64_t(1) << l2;
        const std::vector<std::complex<double>> w1 = roots64(l1), w2 = roots64(l2);
        // t[j1 n2 + j2]: columns j2 (length n1, stride n2)
        auto cols = [&](size_t j2) {
            std::vector<std::complex<double>> c(static_cast<size_t>(n1));
            for (int64_t j1 = 0; j1 < n1; ++j1) c[size_t(j1)] = t[size_t(j1 * n2 + int64_t(j2))];
            fft64_tab(c.data(), l1, w1.data());
            for (int64_t k1 = 0; k1 < n1; ++k1) {
                const double ang = -2.0 * M_PI * double(int64_t(j2) * k1) / double(n);  // w_n^{j2 k1}
                t[size_t(k1 * n2 + int64_t(j2))] = c[size_t(k1)] * std::complex<double>(std::cos(ang), std::sin(ang));
            }
        };
        auto rows = [&](size_t k1) { fft64_tab(t.data() + int64_t(k1) * n2, l2, w2.data()); };
        if (par) {
            parallel_for(size_t(n2), cols);
            parallel_for(size_t(n1), rows);
        } else {
            for (int64_t j2 = 0; j2 < n2; ++j2) cols(size_t(j2));
            for (int64_t k1 = 0; k1 < n1; ++k1) rows(size_t(k1));
        }
        auto put = [&](size_t k2) {
            for (int64_t k1 = 0; k1 < n1; ++k1) a[(k1 + n1 * int64_t(k2)) * stride] = t[size_t(k1 * n2 + int64_t(k2))];
        };
        if (par) parallel_for(size_t(n2), put);
        else for (int64_t k2 = 0; k2 < n2; ++k2) put(size_t(k2));
        return;
    }
    for (int64_t i = 0; i < n; ++i) a[i * stride] = t[size_t(i)];
}

// The recursion of Algorithm 5, level by level: every call of a level is
// decomposed (or, at most s0 vertices, laid out as a dense leaf) independently
// of the others, in parallel when `parallel` is set, and the results are
// appended to the plan in call order, so the plan is the same as a one-call-
// at-a-time breadth-first recursion. Calls of one level hold disjoint vertex
// sets: the vertex-indexed scratch arrays are touched only at a call's own
// members (membership is set for the whole level before it starts), and the
// traversal tokens are unique across threads.
class Builder {
    // vertex-indexed scratch of the traversals; calls of one level use them at
    // their own members only, so one set serves all concurrent calls of a level
    struct Scratch {
        std::vector<int32_t> onp, seen, par;
        std::vector<int64_t> dist, sz, maxchild;
        void init(int32_t n) {
            onp.assign(size_t(n), 0);
            seen.assign(size_t(n), 0);
            par.assign(size_t(n), -1);
            dist.assign(size_t(n), 0);
            sz.assign(size_t(n), 0);
            maxchild.assign(size_t(n), 0);
        }
    };
    static constexpr int64_t kSplitMin = int64_t(1) << 15;  // calls this large build both candidates at once

public:
    Builder(HostPlan &hp, bool parallel) : hp_(hp), n_(hp.n), parallel_(parallel) {
        member_.assign(size_t(n_), 0);
        a_.init(n_);
        // a second set for the centroid branch of large calls (concurrent with the diameter branch)
        if (parallel_ && n_ >= kSplitMin) b_.init(n_);
    }

    int run(std::string &err) {
        // top-level calls: the trees of the forest, in order of their smallest vertex
        std::vector<Item> cur;
        std::fill(member_.begin(), member_.end(), 1);
        std::vector<char> done(size_t(n_), 0);
        std::vector<int32_t> order;
        for (int32_t s = 0; s < n_; ++s) {
            if (done[size_t(s)]) continue;
            traverse(a_, s, 1, order);
            for (int32_t v : order) done[size_t(v)] = 1;
            cur.push_back(Item{0, order, 0});
        }
        int32_t tok_member = 1;
        std::vector<Result> res;
        std::vector<Item> next;
        while (!cur.empty()) {
            for (Item &it : cur) {
                it.mtok = ++tok_member;
                for (int32_t v : it.S) member_[size_t(v)] = it.mtok;
            }
            res.assign(cur.size(), Result{});
            auto one = [&](size_t i) { solve(cur[i], res[i]); };
            if (parallel_) parallel_for(cur.size(), one);
            else for (size_t i = 0; i < cur.size(); ++i) one(i);
            next.clear();
            for (size_t i = 0; i < cur.size(); ++i) {
                const Item &it = cur[i];
                Result &r = res[i];
                hp_.n_levels = std::max(hp_.n_levels, it.level + 1);
                if (r.rc) {
                    err = r.err;
                    return r.rc;
                }
                if (r.leaf) {
                    r.lf.begin = int64_t(hp_.leaf_vtx.size());
                    hp_.leaf_vtx.insert(hp_.leaf_vtx.end(), r.lvtx.begin(), r.lvtx.end());
                    hp_.leaf_dist.insert(hp_.leaf_dist.end(), r.ldist.begin(), r.ldist.end());
                    hp_.leaf_pdist.insert(hp_.leaf_pdist.end(), r.lpdist.begin(), r.lpdist.end());
                    r.lf.end = int64_t(hp_.leaf_vtx.size());
                    hp_.leaves.push_back(r.lf);
                    continue;
                }
                emit_call(it.level, r.minv, int32_t(it.S.size()), r.kind, r.D);
                for (size_t a = 0; a + 1 < r.D.cptr.size(); ++a)
                    next.push_back(Item{it.level + 1,
                                        std::vector<int32_t>(r.D.cv.begin() + r.D.cptr[a], r.D.cv.begin() + r.D.cptr[a + 1]),
                                        0});
            }
            cur.swap(next);
        }
        return TFI_OK;
    }

private:
    struct Item {
        int32_t level;
        std::vector<int32_t> S;
        int32_t mtok;
    };
    struct Result {
        int rc = 0;
        std::string err;
        int32_t minv = 0, kind = 0;
        bool leaf = false;
        Decomp D;
        Leaf lf;
        std::vector<int32_t> lvtx, ldist, lpdist;
    };

    // One call: its decomposition (Algorithm 6 choice, Algorithm 1), or its dense leaf.
    void solve(const Item &it, Result &r) {
        const int32_t mtok = it.mtok;
        const int64_t nS = int64_t(it.S.size());
        r.minv = *std::min_element(it.S.begin(), it.S.end());
        std::vector<int32_t> order;
        if (nS <= hp_.leaf_max) {
            r.leaf = true;
            r.rc = leaf(a_, it.level, r.minv, mtok, r, order);
            return;
        }
        if (hp_.policy == TFI_POLICY_CENTROID) {
            decompose(a_, mtok, {centroid(a_, r.minv, nS, mtok, order)}, r.D);
            r.kind = 1;
        } else if (hp_.policy == TFI_POLICY_DIAMETER) {
            decompose(a_, mtok, diameter(a_, r.minv, mtok, order), r.D);
        } else {
            Decomp dc;
            if (!b_.seen.empty() && nS >= kSplitMin) {
                // both candidates at once, each in its own scratch set
                std::thread th([&]() {
                    std::vector<int32_t> order2;
                    decompose(b_, mtok, {centroid(b_, r.minv, nS, mtok, order2)}, dc);
                });
                decompose(a_, mtok, diameter(a_, r.minv, mtok, order), r.D);
                th.join();
            } else {
                decompose(a_, mtok, diameter(a_, r.minv, mtok, order), r.D);
                decompose(a_, mtok, {centroid(a_, r.minv, nS, mtok, order)}, dc);
            }
            // the centroid wins only with a strictly smaller score (Algorithm 6)
            if (score(nS, dc) < score(nS, r.D)) {
                r.D = std::move(dc);
                r.kind = 1;
            }
        }
        if (r.D.H >= kGridMax || r.D.X.back() >= kGridMax) {
            r.err = "grid distance beyond 2^30 in a decomposition (choose a larger delta)";
            r.rc = TFI_ERR_GRID_OVERFLOW;
        }
    }

    // Traverse the members of S (member == mtok) from s into order: dist_, par_.
    void traverse(Scratch &sc, int32_t s, int32_t mtok, std::vector<int32_t> &order) {
        const int32_t tok = ++tok_seen_;
        order.clear();
        order.push_back(s);
        sc.seen[size_t(s)] = tok;
        sc.dist[size_t(s)] = 0;
        sc.par[size_t(s)] = -1;
        for (size_t h = 0; h < order.size(); ++h) {
            const int32_t a = order[h];
            for (int64_t e = hp_.ptr[size_t(a)]; e < hp_.ptr[size_t(a) + 1]; ++e) {
                const int32_t b = hp_.adj[size_t(e)];
                if (member_[size_t(b)] == mtok && sc.seen[size_t(b)] != tok) {
                    sc.seen[size_t(b)] = tok;
                    sc.dist[size_t(b)] = sc.dist[size_t(a)] + hp_.qlen[size_t(e)];
                    sc.par[size_t(b)] = a;
                    order.push_back(b);
                }
            }
        }
    }

    static int32_t farthest(const Scratch &sc, const std::vector<int32_t> &order) {
        int32_t best = order[0];
        for (int32_t v : order) {
            if (sc.dist[size_t(v)] > sc.dist[size_t(best)] || (sc.dist[size_t(v)] == sc.dist[size_t(best)] && v < best)) best = v;
        }
        return best;
    }

    // Weighted diameter path by two traversals and parent pointers (Algorithm 6, first step).
    std::vector<int32_t> diameter(Scratch &sc, int32_t minv, int32_t mtok, std::vector<int32_t> &order) {
        traverse(sc, minv, mtok, order);
        const int32_t a = farthest(sc, order);
        traverse(sc, a, mtok, order);
        const int32_t b = farthest(sc, order);
        std::vector<int32_t> path;
        for (int32_t v = b; v != -1; v = sc.par[size_t(v)]) path.push_back(v);
        std::reverse(path.begin(), path.end());
        return path;
    }

    // Centroid by a rooted traversal and subtree sizes (Algorithm 6, second step).
    int32_t centroid(Scratch &sc, int32_t minv, int64_t nS, int32_t mtok, std::vector<int32_t> &order) {
        traverse(sc, minv, mtok, order);
        for (int32_t v : order) {
            sc.sz[size_t(v)] = 1;
            sc.maxchild[size_t(v)] = 0;
        }
        for (size_t i = order.size(); i-- > 1;) {
            const int32_t v = order[i], p = sc.par[size_t(v)];
            sc.sz[size_t(p)] += sc.sz[size_t(v)];
            sc.maxchild[size_t(p)] = std::max(sc.maxchild[size_t(p)], sc.sz[size_t(v)]);
        }
        int32_t best = -1;
        for (int32_t v : order) {
            const int64_t big = std::max<int64_t>(nS - sc.sz[size_t(v)], sc.maxchild[size_t(v)]);
            if (2 * big <= nS && (best < 0 || v < best)) best = v;
        }
        return best;
    }

    int64_t edge_len(int32_t a, int32_t b) const {
        for (int64_t e = hp_.ptr[size_t(a)]; e < hp_.ptr[size_t(a) + 1]; ++e)
            if (hp_.adj[size_t(e)] == b) return hp_.qlen[size_t(e)];
        return -1;
    }

    // Algorithm 1: components, anchors, projections and depths for backbone P.
    void decompose(Scratch &sc, int32_t mtok, std::vector<int32_t> P, Decomp &D) {
        D.clear();
        D.P = std::move(P);
        const int32_t ptok = ++tok_onp_;
        for (int32_t p : D.P) sc.onp[size_t(p)] = ptok;
        D.X.push_back(0);
        for (size_t j = 1; j < D.P.size(); ++j) D.X.push_back(D.X.back() + edge_len(D.P[j - 1], D.P[j]));
        const int32_t tok = ++tok_seen_;
        for (size_t j = 0; j < D.P.size(); ++j) {
            const int32_t p = D.P[j];
            for (int64_t e = hp_.ptr[size_t(p)]; e < hp_.ptr[size_t(p) + 1]; ++e) {
                const int32_t r = hp_.adj[size_t(e)];
                if (member_[size_t(r)] != mtok || sc.onp[size_t(r)] == ptok || sc.seen[size_t(r)] == tok) continue;
                const size_t start = D.cv.size();
                sc.seen[size_t(r)] = tok;
                D.cv.push_back(r);
                D.cd.push_back(hp_.qlen[size_t(e)]);  // the attaching edge p - r
                int64_t h = 0;
                for (size_t k = start; k < D.cv.size(); ++k) {
                    const int32_t a = D.cv[k];
                    const int64_t da = D.cd[k];
                    h = std::max(h, da);
                    for (int64_t f = hp_.ptr[size_t(a)]; f < hp_.ptr[size_t(a) + 1]; ++f) {
                        const int32_t b = hp_.adj[size_t(f)];
                        if (member_[size_t(b)] == mtok && sc.onp[size_t(b)] != ptok && sc.seen[size_t(b)] != tok) {
                            sc.seen[size_t(b)] = tok;
                            D.cv.push_back(b);
                            D.cd.push_back(da + hp_.qlen[size_t(f)]);
                        }
                    }
                }
                D.cptr.push_back(int32_t(D.cv.size()));
                D.canchor.push_back(int32_t(j));
                D.cH.push_back(h);
                D.H = std::max(D.H, h);
            }
        }
    }

    // Eq. "stad-score" in grid units, natural log.
    static double score(int64_t nS, const Decomp &D) {
        const double M = double(D.H + 1) * double(D.X.back() + 1);
        double c = double(nS) + M * std::log(std::max(M, 2.0));
        for (int64_t h : D.cH) c += double(h) * std::log(double(h) + 1.0);
        for (size_t a = 0; a + 1 < D.cptr.size(); ++a) {
            const double na = double(D.cptr[a + 1] - D.cptr[a]);
            c += na * std::log(na + 1.0);
        }
        return c;
    }

    void emit_call(int32_t level, int32_t minv, int32_t size, int32_t kind, const Decomp &D) {
        Call c;
        c.level = level;
        c.minv = minv;
        c.size = size;
        c.kind = kind;
        c.bb_begin = int64_t(hp_.bb.size());
        hp_.bb.insert(hp_.bb.end(), D.P.begin(), D.P.end());
        c.bb_end = int64_t(hp_.bb.size());
        c.H = D.H;
        c.L = D.X.back();
        c.rec_begin = int64_t(hp_.recs.size());
        for (size_t j = 0; j < D.P.size(); ++j) hp_.recs.push_back(Rec{D.P[j], 0, int32_t(D.X[j]), -1});
        c.comp_begin = int32_t(hp_.comps.size());
        const int32_t call_idx = int32_t(hp_.calls.size());
        for (size_t a = 0; a + 1 < D.cptr.size(); ++a) {
            const int32_t gid = int32_t(hp_.comps.size());
            Comp cp;
            cp.call = call_idx;
            cp.minv = *std::min_element(D.cv.begin() + D.cptr[a], D.cv.begin() + D.cptr[a + 1]);
            cp.size = D.cptr[a + 1] - D.cptr[a];
            cp.anchor_idx = D.canchor[a];
            cp.H = D.cH[a];
            hp_.comps.push_back(cp);
            const int32_t x = int32_t(D.X[size_t(D.canchor[a])]);
            for (int32_t k = D.cptr[a]; k < D.cptr[a + 1]; ++k)
                hp_.recs.push_back(Rec{D.cv[size_t(k)], int32_t(D.cd[size_t(k)]), x, gid});
        }
        c.comp_end = int32_t(hp_.comps.size());
        c.rec_end = int64_t(hp_.recs.size());
        hp_.calls.push_back(c);
    }

    // Dense leaf: vertices in preorder from the smallest vertex, children ascending,
    // with grid distances from that root (subtrees are contiguous ranges), and the
    // leaf's diameter; begin / end are set when it is appended to the plan.
    int leaf(Scratch &sc, int32_t level, int32_t minv, int32_t mtok, Result &r, std::vector<int32_t> &order) {
        r.lf.level = level;
        r.lf.minv = minv;
        const int32_t tok = ++tok_seen_;
        std::vector<int32_t> stack, kids;
        stack.push_back(minv);
        sc.seen[size_t(minv)] = tok;
        sc.dist[size_t(minv)] = 0;
        sc.par[size_t(minv)] = -1;
        while (!stack.empty()) {
            const int32_t v = stack.back();
            stack.pop_back();
            if (sc.dist[size_t(v)] >= kGridMax / 2) {
                r.err = "grid distance beyond 2^29 inside a leaf (choose a larger delta)";
                return TFI_ERR_GRID_OVERFLOW;
            }
            r.lvtx.push_back(v);
            r.ldist.push_back(int32_t(sc.dist[size_t(v)]));
            const int32_t p = sc.par[size_t(v)];
            r.lpdist.push_back(p >= 0 ? int32_t(sc.dist[size_t(p)]) : 0);
            kids.clear();
            for (int64_t e = hp_.ptr[size_t(v)]; e < hp_.ptr[size_t(v) + 1]; ++e) {
                const int32_t b = hp_.adj[size_t(e)];
                if (member_[size_t(b)] == mtok && sc.seen[size_t(b)] != tok) {
                    sc.seen[size_t(b)] = tok;
                    sc.dist[size_t(b)] = sc.dist[size_t(v)] + hp_.qlen[size_t(e)];
                    sc.par[size_t(b)] = v;
                    kids.push_back(b);
                }
            }
            // adjacency is ascending; push in reverse so the smallest child comes next
            for (size_t k = kids.size(); k-- > 0;) stack.push_back(kids[k]);
        }
        // leaf diameter by a second traversal from the vertex farthest from the root
        int32_t far = minv;
        int64_t best = -1;
        for (size_t i = 0; i < r.lvtx.size(); ++i) {
            if (r.ldist[i] > best) {
                best = r.ldist[i];
                far = r.lvtx[i];
            }
        }
        traverse(sc, far, mtok, order);
        r.lf.diam = 0;
        for (int32_t v : order) r.lf.diam = std::max(r.lf.diam, sc.dist[size_t(v)]);
        return TFI_OK;
    }


    HostPlan &hp_;
    int32_t n_;
    bool parallel_;
    std::vector<int32_t> member_;
    Scratch a_, b_;
    std::atomic<int32_t> tok_onp_{0}, tok_seen_{0};
};

// Cost model of the two evaluators, per channel, in units of one direct
// multiply-add: direct summation touches every key pair; the FFT path pays a
// forward and an inverse transform of the padded table (both halved by packing
// two channels per complex transform) plus the key scatter and read-back.
constexpr double kFftCostPerPointLog = 3.0;
constexpr double kFftCostPerKey = 4.0;
// four-step FFT through global memory: about 22 bytes of DRAM traffic per point and
// channel, against 2 flops per pair and channel for direct summation
constexpr double kBigCostPerPoint = 50.0;
// Hankel evaluator, per occupied backbone column and channel: the split-TF32
// product (NP x KT per channel), the operand staging (KT loads) and two
// prefix-sum updates per row; a CTA always covers 128 channels, so fewer
// channels pay for 128. The weights are calibrated on the attention-width
// workload (12 grid spanning trees of 196 vertices, 4096 channels), where the
// Hankel stage took 0.81x the time of the direct stage over the same tables.
constexpr double kHankelMmaCost = 0.25;
constexpr double kHankelStageCost = 1.0;
constexpr double kHankelScanCost = 3.0;

// Algorithm 7 sweeps, per exponential term and channel: lambda^r weighting in and
// out per bin, one recurrence step per backbone run and direction.
constexpr double kSweepCostPerKey = 6.0;
constexpr double kSweepCostPerRun = 4.0;

double hankel_cost(int32_t H, int32_t L, double ncols, double nk, int d) {
    const HankelLayout lay = hankel_layout(H, L);
    const double per_col = kHankelMmaCost * lay.NP * lay.KT + kHankelStageCost * lay.KT + kHankelScanCost * lay.S;
    return ncols * per_col * 128.0 / double(std::min(d, 128)) + 2 * nk;
}


// 1 + the largest k < len whose FP32 sample float(f(k delta)) is not zero (0 if none): every
// sample from there to len - 1 is zero. Scanned downwards in chunks on all host threads.
int64_t fp32_support(const KernelFn &f, double delta, int64_t len) {
    constexpr int64_t kChunk = int64_t(1) << 16;
    const size_t nch = size_t((len + kChunk - 1) / kChunk);
    std::vector<int64_t> last(nch, -1);
    parallel_for(nch, [&](size_t c) {
        const int64_t lo = int64_t(c) * kChunk, hi = std::min(len, lo + kChunk);
        for (int64_t k = hi - 1; k >= lo; --k)
            if (float(f.grid(k, delta)) != 0.f) {
                last[c] = k;
                return;
            }
    });
    for (size_t c = nch; c-- > 0;)
        if (last[c] >= 0) return last[c] + 1;
    return 0;
}

// Bins of one call: its A-bins (distinct (depth, coordinate)) and each
// component's b-bins (distinct depth), members ascending by vertex id.
struct CallBins {
    std::vector<int32_t> kr, kx, ksize, kvtx;   // bins in order; member lists concatenated
    std::vector<int32_t> rec_akey, rec_bkey;    // per record of the call (local bin index, -1 none)
    std::vector<std::pair<int32_t, int32_t>> jobs;  // local bin ranges: call table first, then components
};

void build_call_bins(const HostPlan &hp, const Call &call, CallBins &cb) {
    const int64_t nrec = call.rec_end - call.rec_begin;
    cb.rec_akey.assign(size_t(nrec), -1);
    cb.rec_bkey.assign(size_t(nrec), -1);
    struct Item {
        uint64_t key;
        int32_t v;
        int32_t pos;
        bool operator<(const Item &o) const { return key != o.key ? key < o.key : v < o.v; }
    };
    std::vector<Item> items(static_cast<size_t>(nrec));
    for (int64_t i = 0; i < nrec; ++i) {
        const Rec &rc = hp.recs[size_t(call.rec_begin + i)];
        items[size_t(i)] = Item{(uint64_t(uint32_t(rc.r)) << 32) | uint32_t(rc.x), rc.v, int32_t(i)};
    }
    std::sort(items.begin(), items.end());
    int32_t kb = 0;
    for (size_t i = 0; i < items.size(); ++i) {
        if (i == 0 || items[i].key != items[i - 1].key) {
            cb.kr.push_back(int32_t(items[i].key >> 32));
            cb.kx.push_back(int32_t(items[i].key & 0xffffffffu));
            cb.ksize.push_back(0);
        }
        cb.ksize.back()++;
        cb.kvtx.push_back(items[i].v);
        cb.rec_akey[size_t(items[i].pos)] = int32_t(cb.kr.size() - 1);
    }
    cb.jobs.push_back({kb, int32_t(cb.kr.size())});
    int64_t pos = call.bb_end - call.bb_begin;
    for (int32_t a = call.comp_begin; a < call.comp_end; ++a) {
        const int64_t cbeg = pos, cend = pos + hp.comps[size_t(a)].size;
        pos = cend;
        items.resize(size_t(cend - cbeg));
        for (int64_t i = cbeg; i < cend; ++i) {
            const Rec &rc = hp.recs[size_t(call.rec_begin + i)];
            items[size_t(i - cbeg)] = Item{uint64_t(uint32_t(rc.r)), rc.v, int32_t(i)};
        }
        std::sort(items.begin(), items.end());
        kb = int32_t(cb.kr.size());
        for (size_t i = 0; i < items.size(); ++i) {
            if (i == 0 || items[i].key != items[i - 1].key) {
                cb.kr.push_back(int32_t(items[i].key));
                cb.kx.push_back(0);
                cb.ksize.push_back(0);
            }
            cb.ksize.back()++;
            cb.kvtx.push_back(items[i].v);
            cb.rec_bkey[size_t(items[i].pos)] = int32_t(cb.kr.size() - 1);
        }
        cb.jobs.push_back({kb, int32_t(cb.kr.size())});
    }
}

}  // namespace

// Everything in a plan that depends on the values of f: FP32 grid samples, the
// FP64-computed spectra of kappa[j][b] = f(j + min(b, P2 - b)) per FFT size
// class (scaled by 1/(P1 P2), bit-reversed along both axes), and the terms of
// an exponential sum for the sweeps.
int sample_kernel(HostPlan &hp, std::string &err) {
    if (hp.f.kind == TFI_F_TABLE && hp.hist_len > int64_t(hp.f.table.size())) {
        err = "sampled kernel table shorter than the largest grid distance the plan needs";
        return TFI_ERR_GRID_OVERFLOW;
    }
    if (hp.trunc >= 0 && fp32_support(hp.f, hp.delta, hp.trunc_check) > hp.trunc) {
        err = "the kernel's FP32 samples reach beyond the distance at which the plan truncated its tables; plan again";
        return TFI_ERR_UNSUPPORTED;
    }
    hp.ftab.resize(size_t(hp.ftab_len));
    for (int64_t k = 0; k < hp.ftab_len; ++k) hp.ftab[size_t(k)] = float(hp.f.grid(k, hp.delta));
    std::vector<std::complex<double>> buf;
    for (int cls = 0; cls < kSpecClasses; ++cls) {
        const int64_t off = hp.spec_class_off[size_t(cls)];
        if (off < 0) continue;
        const int lp1 = cls / 32, lp2 = cls % 32;
        const int64_t P1 = int64_t(1) << lp1, P2 = int64_t(1) << lp2, NP = P1 * P2;
        const bool big = lp1 + lp2 > kFftMaxLog;
        buf.assign(size_t(NP), 0.0);
        auto fill_row = [&](size_t a) {
            for (int64_t b = 0; b < P2; ++b) {
                double fv = hp.f.grid(int64_t(a) + std::min(b, P2 - b), hp.delta);
                if (!std::isfinite(fv)) fv = 0.0;  // beyond a sampled table: never read for occupied bins
                buf[size_t(int64_t(a) * P2 + b)] = fv;
            }
        };
        auto fft_row = [&](size_t a) { fft64_any(buf.data() + int64_t(a) * P2, lp2, 1, false); };
        auto fft_col = [&](size_t b) { fft64_any(buf.data() + int64_t(b), lp1, P2, big && P2 == 1); };
        if (big) {
            // rows in chunks of at least 2^12 points per task
            const int64_t rows_per = std::max<int64_t>(1, (int64_t(1) << 12) / P2);
            parallel_for(size_t((P1 + rows_per - 1) / rows_per), [&](size_t c) {
                for (int64_t a = int64_t(c) * rows_per; a < std::min(P1, int64_t(c + 1) * rows_per); ++a) fill_row(size_t(a));
            });
            if (lp2 > 0) parallel_for(size_t(P1), fft_row);
            if (P2 > 1) parallel_for(size_t(P2), fft_col);
            else fft_col(0);
        } else {
            for (int64_t a = 0; a < P1; ++a) fill_row(size_t(a));
            for (int64_t a = 0; a < P1; ++a) fft_row(size_t(a));
            for (int64_t b = 0; b < P2; ++b) fft_col(size_t(b));
        }
        const double scale = 1.0 / double(NP);
        float *dst = hp.spectra.data() + off;
        if (!big) {
            // slot (a, b) holds frequency (brev a, brev b): the order the shared-memory FFT leaves
            for (int64_t a = 0; a < P1; ++a) {
                for (int64_t b = 0; b < P2; ++b) {
                    const std::complex<double> sv =
                        buf[size_t(int64_t(bitrev(uint32_t(a), lp1)) * P2 + int64_t(bitrev(uint32_t(b), lp2)))] * scale;
                    dst[2 * (a * P2 + b)] = float(sv.real());
                    dst[2 * (a * P2 + b) + 1] = float(sv.imag());
                }
            }
        } else {
            // four-step order: slot s BLK + sb P2 + sc (column-FFT slot s, block slots sb, sc) holds
            // outer frequency brev(s) + N1a brev(sb) and inner frequency brev(sc)
            const BigSplit sp = big_split(lp1, lp2);
            const int64_t NA = int64_t(1) << sp.lnA, NB = int64_t(1) << sp.lp1b, BLK = NB * P2;
            parallel_for(size_t(NA), [&](size_t si) {
                const int64_t s = int64_t(si);
                const int64_t ka = bitrev(uint32_t(s), sp.lnA);
                for (int64_t sb = 0; sb < NB; ++sb) {
                    const int64_t k1 = ka + NA * int64_t(bitrev(uint32_t(sb), sp.lp1b));
                    for (int64_t sc = 0; sc < P2; ++sc) {
                        const std::complex<double> sv = buf[size_t(k1 * P2 + int64_t(bitrev(uint32_t(sc), lp2)))] * scale;
                        const int64_t pos = s * BLK + sb * P2 + sc;
                        dst[2 * pos] = float(sv.real());
                        dst[2 * pos + 1] = float(sv.imag());
                    }
                }
            });
        }
    }
    hp.sw_coef.clear();
    hp.sw_beta.clear();
    if ((hp.flags & (TFI_PLAN_SWEEP | TFI_PLAN_SWEEP_AUTO)) && hp.f.kind == TFI_F_EXPSUM) {
        for (size_t i = 0; i + 1 < hp.f.params.size(); i += 2) {
            hp.sw_coef.push_back(float(hp.f.params[i]));
            hp.sw_beta.push_back(float(hp.f.params[i + 1] * hp.delta));
        }
    }
    return TFI_OK;
}

namespace {

// roots: the smallest vertex of each tree of the forest
int flatten(HostPlan &hp, const std::vector<int32_t> &roots, std::string &err) {
    const int64_t R = int64_t(hp.recs.size());
    std::vector<int32_t> rec_akey(size_t(R), -1), rec_bkey(size_t(R), -1);
    const size_t C = hp.calls.size();
    // bins per call, in parallel; then global offsets in call order
    std::vector<CallBins> bins(C);
    parallel_for(C, [&](size_t c) { build_call_bins(hp, hp.calls[c], bins[c]); });
    std::vector<int64_t> koff(C + 1, 0), voff(C + 1, 0), joff(C + 1, 0);
    for (size_t c = 0; c < C; ++c) {
        koff[c + 1] = koff[c] + int64_t(bins[c].kr.size());
        voff[c + 1] = voff[c] + int64_t(bins[c].kvtx.size());
        joff[c + 1] = joff[c] + int64_t(bins[c].jobs.size());
    }
    if (voff[C] >= int64_t(INT32_MAX)) {
        err = "plan too large for 32-bit bin indices";
        return TFI_ERR_UNSUPPORTED;
    }
    // support truncation (not with the exponential sweeps, whose jobs span whole calls)
    hp.trunc = -1;
    hp.zero_ranges.clear();
    hp.jobs_full.clear();
    {
        int64_t need_calls = 0;
        for (const Call &c : hp.calls) need_calls = std::max<int64_t>(need_calls, 2 * c.H + c.L);
        hp.trunc_check = need_calls + 1;
        if (!(hp.flags & (TFI_PLAN_SWEEP | TFI_PLAN_SWEEP_AUTO | TFI_PLAN_NO_TRUNCATE)) && !hp.calls.empty()) {
            const int64_t T = fp32_support(hp.f, hp.delta, hp.trunc_check);
            if (T < hp.trunc_check) hp.trunc = T;
        }
    }
    std::vector<std::vector<int32_t>> call_zero(hp.trunc >= 0 ? C : 0);
    if (hp.trunc >= 0) hp.jobs_full.resize(size_t(joff[C]));
    hp.key_r.resize(size_t(koff[C]));
    hp.key_x.resize(size_t(koff[C]));
    hp.key_ptr.resize(size_t(koff[C]) + 1);
    hp.key_vtx.resize(size_t(voff[C]));
    hp.jobs.resize(size_t(joff[C]));
    hp.key_ptr[size_t(koff[C])] = int32_t(voff[C]);
    parallel_for(C, [&](size_t c) {
        CallBins &cb = bins[c];
        const Call &call = hp.calls[c];
        int64_t vo = voff[c];
        for (size_t k = 0; k < cb.kr.size(); ++k) {
            hp.key_r[size_t(koff[c]) + k] = cb.kr[k];
            hp.key_x[size_t(koff[c]) + k] = cb.kx[k];
            hp.key_ptr[size_t(koff[c]) + k] = int32_t(vo);
            vo += cb.ksize[k];
        }
        std::copy(cb.kvtx.begin(), cb.kvtx.end(), hp.key_vtx.begin() + voff[c]);
        for (int64_t i = 0; i < call.rec_end - call.rec_begin; ++i) {
            rec_akey[size_t(call.rec_begin + i)] = int32_t(koff[c]) + cb.rec_akey[size_t(i)];
            if (cb.rec_bkey[size_t(i)] >= 0)
                rec_bkey[size_t(call.rec_begin + i)] = int32_t(koff[c]) + cb.rec_bkey[size_t(i)];
        }
        for (size_t j = 0; j < cb.jobs.size(); ++j) {
            Job jb{};
            jb.kb = koff[c] + cb.jobs[j].first;
            jb.ke = koff[c] + cb.jobs[j].second;
            jb.is_comp = j > 0 ? 1 : 0;
            if (hp.trunc >= 0) {
                // the untruncated job (for the kernel gradient), then the cut: bins ascend in depth,
                // and those at depth >= trunc only read zero samples
                Job full = jb;
                for (int64_t k = full.kb; k < full.ke; ++k) {
                    full.maxr = std::max(full.maxr, hp.key_r[size_t(k)]);
                    full.maxx = std::max(full.maxx, hp.key_x[size_t(k)]);
                }
                full.lp1 = ceil_log2(2 * int64_t(full.maxr) + 1);
                full.lp2 = full.maxx > 0 ? ceil_log2(2 * int64_t(full.maxx)) : 0;
                hp.jobs_full[size_t(joff[c]) + j] = full;
                int64_t cut = jb.kb;
                while (cut < jb.ke && hp.key_r[size_t(cut)] < hp.trunc) ++cut;
                if (cut < jb.ke) call_zero[c].insert(call_zero[c].end(), {int32_t(cut), int32_t(jb.ke)});
                jb.ke = cut;
            }
            int32_t maxr = 0, maxx = 0;
            for (int64_t k = jb.kb; k < jb.ke; ++k) {
                maxr = std::max(maxr, hp.key_r[size_t(k)]);
                maxx = std::max(maxx, hp.key_x[size_t(k)]);
            }
            jb.maxr = maxr;
            jb.maxx = maxx;
            jb.lp1 = ceil_log2(2 * int64_t(maxr) + 1);
            jb.lp2 = maxx > 0 ? ceil_log2(2 * int64_t(maxx)) : 0;
            const double nk = double(jb.ke - jb.kb);
            const int lg = jb.lp1 + jb.lp2;
            const double np = std::ldexp(1.0, lg);
            const double cost_fft = kFftCostPerPointLog * np * std::max(1, lg) + kFftCostPerKey * nk;
            const bool fft_ok = lg <= kFftMaxLog && !(hp.flags & TFI_PLAN_DIRECT_ALL);
            jb.mode = (fft_ok && cost_fft < nk * nk) ? 0 : 1;
            double best = jb.mode == 0 ? cost_fft : nk * nk;
            // tables beyond shared memory: the four-step FFT through global memory, which also
            // pays for its passes over the whole padded table in DRAM
            if (!fft_ok && !(hp.flags & TFI_PLAN_DIRECT_ALL) && lg <= kBigMaxLog && jb.lp2 <= kBigMaxInnerLog &&
                jb.lp1 >= 1) {
                const double cost_big = kFftCostPerPointLog * np * lg + kBigCostPerPoint * np + kFftCostPerKey * nk;
                if (cost_big < best || (hp.flags & TFI_PLAN_FFT_BIG_ALL)) {
                    jb.mode = 4;
                    best = cost_big;
                }
            }
            // occupied backbone columns (runs of equal coordinate)
            int64_t ncols = 0;
            if ((hp.flags & (TFI_PLAN_HANKEL | TFI_PLAN_HANKEL_ALL | TFI_PLAN_SWEEP_AUTO))) {
                std::vector<int32_t> xs(hp.key_x.begin() + jb.kb, hp.key_x.begin() + jb.ke);
                std::sort(xs.begin(), xs.end());
                ncols = int64_t(std::unique(xs.begin(), xs.end()) - xs.begin());
            }
            const bool hk_ok = (hp.flags & (TFI_PLAN_HANKEL | TFI_PLAN_HANKEL_ALL)) && hankel_fits(maxr, maxx);
            if (hk_ok) {
                const double ch = hankel_cost(maxr, maxx, double(ncols), nk, hp.max_channels);
                if ((hp.flags & TFI_PLAN_HANKEL_ALL) || ch < best) {
                    jb.mode = 3;
                    best = ch;
                }
            }
            if ((hp.flags & TFI_PLAN_SWEEP_AUTO) && hp.f.kind == TFI_F_EXPSUM) {
                const double J = double(hp.f.params.size() / 2);
                if (J * (kSweepCostPerKey * nk + kSweepCostPerRun * double(ncols)) < best) jb.mode = 2;
            }
            hp.jobs[size_t(joff[c]) + j] = jb;
        }
        CallBins().kr.swap(cb.kr);
        cb = CallBins();
    });
    for (const std::vector<int32_t> &z : call_zero) hp.zero_ranges.insert(hp.zero_ranges.end(), z.begin(), z.end());
    if (hp.zero_ranges.empty()) {
        // no bin lies beyond the support: the tables are whole, and any kernel may replace f later
        hp.trunc = -1;
        hp.jobs_full.clear();
    }
    if (hp.flags & TFI_PLAN_SWEEP) {
        // Algorithm 7 for every table
        for (Job &j : hp.jobs) j.mode = 2;
    }
    {
        // one sweep job per call whose cross table is evaluated by the sweeps (its
        // components' corrections are separate jobs, swept or not by their own mode)
        for (size_t c = 0; c < C; ++c) {
            const Job &g = hp.jobs[size_t(joff[c])];
            if (g.mode != 2) continue;
            SweepJob sj{};
            sj.sb = int32_t(hp.sw_keys.size());
            std::vector<int32_t> ks(size_t(g.ke - g.kb));
            std::iota(ks.begin(), ks.end(), int32_t(g.kb));
            std::stable_sort(ks.begin(), ks.end(), [&](int32_t a, int32_t b) {
                return hp.key_x[size_t(a)] != hp.key_x[size_t(b)] ? hp.key_x[size_t(a)] < hp.key_x[size_t(b)]
                                                                  : hp.key_r[size_t(a)] < hp.key_r[size_t(b)];
            });
            sj.rb = int32_t(hp.sw_run.size());
            for (size_t i = 0; i < ks.size(); ++i) {
                if (i == 0 || hp.key_x[size_t(ks[i])] != hp.key_x[size_t(ks[i - 1])])
                    hp.sw_run.push_back(int32_t(hp.sw_keys.size()));
                hp.sw_keys.push_back(ks[i]);
            }
            sj.se = int32_t(hp.sw_keys.size());
            sj.m = int32_t(hp.sw_run.size()) - sj.rb;
            hp.sw_run.push_back(sj.se);  // closing boundary of the last run
            sj.cjb = int32_t(joff[c] + 1);
            sj.cje = int32_t(joff[c + 1]);
            hp.sweeps.push_back(sj);
        }
    }
    if (hp.key_vtx.size() >= size_t(INT32_MAX)) {
        err = "plan too large for 32-bit bin indices";
        return TFI_ERR_UNSUPPORTED;
    }
    // per vertex: its (A-key, b-key) in every non-leaf call, in level order
    // (a counting sort by vertex, stable in record order: slots are claimed in any
    // order in parallel, then each vertex's few slots are put back in record order)
    hp.vrec_ptr.assign(size_t(hp.n) + 1, 0);
    constexpr int64_t kRecBlock = int64_t(1) << 16;
    const size_t nrb = size_t((R + kRecBlock - 1) / kRecBlock);
    {
        std::vector<std::atomic<int32_t>> cnt(size_t(hp.n));
        for (auto &c : cnt) c.store(0, std::memory_order_relaxed);
        parallel_for(nrb, [&](size_t b) {
            const int64_t i1 = std::min(R, int64_t(b + 1) * kRecBlock);
            for (int64_t i = int64_t(b) * kRecBlock; i < i1; ++i)
                cnt[size_t(hp.recs[size_t(i)].v)].fetch_add(1, std::memory_order_relaxed);
        });
        for (int32_t v = 0; v < hp.n; ++v)
            hp.vrec_ptr[size_t(v) + 1] = hp.vrec_ptr[size_t(v)] + cnt[size_t(v)].load(std::memory_order_relaxed);
        for (int32_t v = 0; v < hp.n; ++v) cnt[size_t(v)].store(hp.vrec_ptr[size_t(v)], std::memory_order_relaxed);
        std::vector<int32_t> rec_of(static_cast<size_t>(R));
        parallel_for(nrb, [&](size_t b) {
            const int64_t i1 = std::min(R, int64_t(b + 1) * kRecBlock);
            for (int64_t i = int64_t(b) * kRecBlock; i < i1; ++i)
                rec_of[size_t(cnt[size_t(hp.recs[size_t(i)].v)].fetch_add(1, std::memory_order_relaxed))] = int32_t(i);
        });
        hp.vrec_akey.assign(size_t(R), 0);
        hp.vrec_bkey.assign(size_t(R), 0);
        constexpr int32_t kVBlock = 1 << 14;
        parallel_for(size_t((hp.n + kVBlock - 1) / kVBlock), [&](size_t b) {
            const int32_t v0 = int32_t(b) * kVBlock, v1 = std::min(hp.n, v0 + kVBlock);
            for (int32_t v = v0; v < v1; ++v) {
                const int32_t s0 = hp.vrec_ptr[size_t(v)], s1 = hp.vrec_ptr[size_t(v) + 1];
                std::sort(rec_of.begin() + s0, rec_of.begin() + s1);
                for (int32_t k = s0; k < s1; ++k) {
                    hp.vrec_akey[size_t(k)] = rec_akey[size_t(rec_of[size_t(k)])];
                    hp.vrec_bkey[size_t(k)] = rec_bkey[size_t(rec_of[size_t(k)])];
                }
            }
        });
    }
    // rooted forest for the device distance pass: each tree rooted at its smallest
    // vertex (parent, edge length and hop depth do not depend on the traversal order,
    // so the trees are traversed in parallel)
    {
        hp.k1_parent.assign(size_t(hp.n), -1);
        hp.k1_qpar.assign(size_t(hp.n), 0);
        std::vector<int32_t> hop(size_t(hp.n), 0);
        std::vector<int32_t> tree_maxhop(roots.size(), 0);
        parallel_for(roots.size(), [&](size_t t) {
            const int32_t s0 = roots[t];
            std::vector<int32_t> queue{s0};
            hp.k1_parent[size_t(s0)] = s0;
            int32_t mh = 0;
            for (size_t h = 0; h < queue.size(); ++h) {
                const int32_t a = queue[h];
                for (int64_t e = hp.ptr[size_t(a)]; e < hp.ptr[size_t(a) + 1]; ++e) {
                    const int32_t b = hp.adj[size_t(e)];
                    if (hp.k1_parent[size_t(b)] >= 0) continue;
                    hp.k1_parent[size_t(b)] = a;
                    hp.k1_qpar[size_t(b)] = int32_t(hp.qlen[size_t(e)]);
                    hop[size_t(b)] = hop[size_t(a)] + 1;
                    mh = std::max(mh, hop[size_t(b)]);
                    queue.push_back(b);
                }
            }
            tree_maxhop[t] = mh;
        });
        for (int32_t mh : tree_maxhop) hp.k1_maxhop = std::max(hp.k1_maxhop, mh);
        hp.rec_anchor.resize(hp.recs.size());
        hp.rec_p1.resize(hp.recs.size());
        parallel_for(hp.calls.size(), [&](size_t ci) {
            const Call &c = hp.calls[ci];
            const int32_t p1 = hp.bb[size_t(c.bb_begin)];
            for (int64_t i = c.rec_begin; i < c.rec_end; ++i) {
                const Rec &rc = hp.recs[size_t(i)];
                hp.rec_anchor[size_t(i)] =
                    rc.comp >= 0 ? hp.bb[size_t(c.bb_begin + hp.comps[size_t(rc.comp)].anchor_idx)] : rc.v;
                hp.rec_p1[size_t(i)] = p1;
            }
        });
    }
    hp.in_leaf.assign(size_t(hp.n), 0);
    for (int32_t v : hp.leaf_vtx) hp.in_leaf[size_t(v)] = 1;
    // leaf groups
    hp.lgrp_ptr.assign(1, 0);
    hp.leaf_lo.assign(hp.leaf_vtx.size(), 0);
    hp.leaf_hi.assign(hp.leaf_vtx.size(), 0);
    int64_t gstart = 0;
    int64_t need_leaf = 0;
    for (const Leaf &lf : hp.leaves) {
        if (lf.end - gstart > kLeafGroup && lf.begin > gstart) {
            hp.lgrp_ptr.push_back(int32_t(lf.begin));
            gstart = lf.begin;
        }
        for (int64_t i = lf.begin; i < lf.end; ++i) {
            hp.leaf_lo[size_t(i)] = int32_t(lf.begin);
            hp.leaf_hi[size_t(i)] = int32_t(lf.end);
        }
        need_leaf = std::max<int64_t>(need_leaf, lf.diam);
    }
    if (int64_t(hp.leaf_vtx.size()) > gstart) hp.lgrp_ptr.push_back(int32_t(hp.leaf_vtx.size()));
    // grid samples of f: every direct job and leaf looks values up by index
    int64_t need = need_leaf;
    int64_t need_any = need_leaf;
    for (const Job &j : hp.jobs) {
        const int64_t top = 2 * int64_t(j.maxr) + j.maxx;
        need_any = std::max(need_any, top);
        if (j.mode == 1 || j.mode == 3) need = std::max(need, top);
    }
    for (const Job &j : hp.jobs_full) need_any = std::max<int64_t>(need_any, 2 * int64_t(j.maxr) + j.maxx);
    hp.ftab_len = need + 1;
    hp.leaf_ftab_len = need_leaf + 1;
    hp.hist_len = std::max(need_any, need_leaf) + 1;
    // FFT size classes in first-use order; their spectra depend on f
    hp.spec_class_off.assign(kSpecClasses, -1);
    int64_t off = 0;
    for (const Job &j : hp.jobs) {
        if (j.mode != 0 && j.mode != 4) continue;
        const int cls = j.lp1 * 32 + j.lp2;
        if (hp.spec_class_off[size_t(cls)] >= 0) continue;
        hp.spec_class_off[size_t(cls)] = off;
        off += int64_t(2) << (j.lp1 + j.lp2);
    }
    hp.spectra.assign(size_t(off), 0.f);
    if (int rc = sample_kernel(hp, err)) return rc;
    // compact per-level twiddles: twiddle[h + o] = exp(-2 pi i o / (8 h)) for h = 2^L, o < h
    const int64_t tw = int64_t(1) << kTwLog;
    hp.twiddle.assign(size_t(2 * tw), 0.f);
    for (int64_t h = 1; h < tw; h <<= 1) {
        for (int64_t o = 0; o < h; ++o) {
            const double ang = -2.0 * M_PI * double(o) / double(8 * h);
            hp.twiddle[size_t(2 * (h + o))] = float(std::cos(ang));
            hp.twiddle[size_t(2 * (h + o) + 1)] = float(std::sin(ang));
        }
    }
    return TFI_OK;
}

// Plan every tree of a forest on its own, in parallel, with an order-preserving
// local relabelling (local id = rank of the vertex id within its tree, so every
// smallest-id tie-break is unchanged), then merge the per-tree plans in tree
// order. Each vertex belongs to one tree, so per-vertex call order (level order)
// and every bin's member order are the same as planning the forest as a whole.
int plan_forest(HostPlan &hp, const std::vector<std::vector<int32_t>> &trees, std::string &err) {
    const size_t T = trees.size();
    std::vector<HostPlan> local(T);
    std::vector<std::string> errs(T);
    std::vector<int> rcs(T, 0);
    std::vector<size_t> order(T);
    std::iota(order.begin(), order.end(), size_t(0));
    std::sort(order.begin(), order.end(), [&](size_t a, size_t b) { return trees[a].size() > trees[b].size(); });
    std::atomic<size_t> next(0);
    auto worker = [&]() {
        std::vector<int32_t> loc_of;  // global -> local, filled per tree
        for (;;) {
            const size_t qi = next.fetch_add(1);
            if (qi >= T) break;
            const size_t t = order[qi];
            const std::vector<int32_t> &vs = trees[t];
            HostPlan &lp = local[t];
            lp.n = int32_t(vs.size());
            lp.delta = hp.delta;
            lp.f = hp.f;
            lp.policy = hp.policy;
            lp.leaf_max = hp.leaf_max;
            lp.ptr.assign(vs.size() + 1, 0);
            for (size_t i = 0; i < vs.size(); ++i) lp.ptr[i + 1] = lp.ptr[i] + (hp.ptr[size_t(vs[i]) + 1] - hp.ptr[size_t(vs[i])]);
            lp.adj.resize(size_t(lp.ptr.back()));
            lp.qlen.resize(size_t(lp.ptr.back()));
            for (size_t i = 0; i < vs.size(); ++i) {
                int64_t o = lp.ptr[i];
                for (int64_t e = hp.ptr[size_t(vs[i])]; e < hp.ptr[size_t(vs[i]) + 1]; ++e, ++o) {
                    const int32_t g = hp.adj[size_t(e)];
                    lp.adj[size_t(o)] = int32_t(std::lower_bound(vs.begin(), vs.end(), g) - vs.begin());
                    lp.qlen[size_t(o)] = hp.qlen[size_t(e)];
                }
            }
            Builder b(lp, false);
            rcs[t] = b.run(errs[t]);
            lp.ptr.clear();
            lp.ptr.shrink_to_fit();
            lp.adj.clear();
            lp.adj.shrink_to_fit();
            lp.qlen.clear();
            lp.qlen.shrink_to_fit();
        }
    };
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const size_t nth = std::min<size_t>(T, hw);
    std::vector<std::thread> pool;
    for (size_t i = 1; i < nth; ++i) pool.emplace_back(worker);
    worker();
    for (std::thread &th : pool) th.join();
    for (size_t t = 0; t < T; ++t) {
        if (rcs[t]) {
            err = errs[t];
            return rcs[t];
        }
    }
    // merge in tree order, mapping local ids back to global ones: offsets of each
    // tree's part by prefix sums, then the trees copied in parallel
    struct Off {
        int64_t call, bb, rec, comp, leaf, lv;
    };
    std::vector<Off> off(T + 1, Off{0, 0, 0, 0, 0, 0});
    for (size_t t = 0; t < T; ++t) {
        const HostPlan &lp = local[t];
        off[t + 1] = Off{off[t].call + int64_t(lp.calls.size()), off[t].bb + int64_t(lp.bb.size()),
                         off[t].rec + int64_t(lp.recs.size()), off[t].comp + int64_t(lp.comps.size()),
                         off[t].leaf + int64_t(lp.leaves.size()), off[t].lv + int64_t(lp.leaf_vtx.size())};
        hp.n_levels = std::max(hp.n_levels, lp.n_levels);
    }
    hp.calls.resize(size_t(off[T].call));
    hp.bb.resize(size_t(off[T].bb));
    hp.recs.resize(size_t(off[T].rec));
    hp.comps.resize(size_t(off[T].comp));
    hp.leaves.resize(size_t(off[T].leaf));
    hp.leaf_vtx.resize(size_t(off[T].lv));
    hp.leaf_dist.resize(size_t(off[T].lv));
    hp.leaf_pdist.resize(size_t(off[T].lv));
    parallel_for(T, [&](size_t t) {
        const std::vector<int32_t> &vs = trees[t];
        HostPlan &lp = local[t];
        const Off &o = off[t];
        for (size_t i = 0; i < lp.calls.size(); ++i) {
            Call c = lp.calls[i];
            c.minv = vs[size_t(c.minv)];
            c.bb_begin += o.bb;
            c.bb_end += o.bb;
            c.rec_begin += o.rec;
            c.rec_end += o.rec;
            c.comp_begin += int32_t(o.comp);
            c.comp_end += int32_t(o.comp);
            hp.calls[size_t(o.call) + i] = c;
        }
        for (size_t i = 0; i < lp.bb.size(); ++i) hp.bb[size_t(o.bb) + i] = vs[size_t(lp.bb[i])];
        for (size_t i = 0; i < lp.recs.size(); ++i) {
            Rec r = lp.recs[i];
            r.v = vs[size_t(r.v)];
            if (r.comp >= 0) r.comp += int32_t(o.comp);
            hp.recs[size_t(o.rec) + i] = r;
        }
        for (size_t i = 0; i < lp.comps.size(); ++i) {
            Comp cp = lp.comps[i];
            cp.call += int32_t(o.call);
            cp.minv = vs[size_t(cp.minv)];
            hp.comps[size_t(o.comp) + i] = cp;
        }
        for (size_t i = 0; i < lp.leaves.size(); ++i) {
            Leaf lf = lp.leaves[i];
            lf.minv = vs[size_t(lf.minv)];
            lf.begin += o.lv;
            lf.end += o.lv;
            hp.leaves[size_t(o.leaf) + i] = lf;
        }
        for (size_t i = 0; i < lp.leaf_vtx.size(); ++i) {
            hp.leaf_vtx[size_t(o.lv) + i] = vs[size_t(lp.leaf_vtx[i])];
            hp.leaf_dist[size_t(o.lv) + i] = lp.leaf_dist[i];
            hp.leaf_pdist[size_t(o.lv) + i] = lp.leaf_pdist[i];
        }
        lp = HostPlan();
    });
    return TFI_OK;
}

}  // namespace

int build_plan(HostPlan &hp, int32_t n, int32_t m, const int32_t *u, const int32_t *v, const double *w,
               std::string &err) {
    const auto t0 = std::chrono::steady_clock::now();
    hp.n = n;
    // validate and quantise: q_e = max(1, round(w_e / delta)), ties to even; in
    // blocks of edges, reporting the first failing edge as a serial pass would
    std::vector<int64_t> q(static_cast<size_t>(m));
    {
        constexpr int32_t kEdgeBlock = 1 << 16;
        const size_t nb = size_t((int64_t(m) + kEdgeBlock - 1) / kEdgeBlock);
        std::vector<int32_t> bad_edge(nb, -1), bad_code(nb, 0);
        parallel_for(nb, [&](size_t b) {
            const int32_t i0 = int32_t(b) * kEdgeBlock, i1 = std::min(m, i0 + kEdgeBlock);
            for (int32_t i = i0; i < i1; ++i) {
                int code = 0;
                double r = 0.0;
                if (u[i] < 0 || u[i] >= n || v[i] < 0 || v[i] >= n || u[i] == v[i]) {
                    code = TFI_ERR_NOT_TREE;
                } else if (!std::isfinite(w[i]) || !(w[i] > 0.0)) {
                    code = TFI_ERR_WEIGHT;
                } else {
                    r = std::nearbyint(w[i] / hp.delta);
                    if (!(r < double(kGridMax))) code = TFI_ERR_GRID_OVERFLOW;
                }
                if (code) {
                    bad_edge[b] = i;
                    bad_code[b] = code;
                    return;
                }
                q[size_t(i)] = std::max<int64_t>(1, int64_t(r));
            }
        });
        for (size_t b = 0; b < nb; ++b) {
            if (bad_edge[b] < 0) continue;
            const int32_t i = bad_edge[b];
            if (bad_code[b] == TFI_ERR_NOT_TREE)
                err = "edge " + std::to_string(i) + " has an out-of-range endpoint or is a self loop";
            else if (bad_code[b] == TFI_ERR_WEIGHT)
                err = "edge " + std::to_string(i) + " has a weight that is not finite and positive";
            else
                err = "edge length / delta exceeds 2^30";
            return bad_code[b];
        }
    }
    // acyclicity by union-find (a forest on n vertices); the sets are the trees
    std::vector<int32_t> par(static_cast<size_t>(n));
    std::iota(par.begin(), par.end(), 0);
    auto find = [&](int32_t a) {
        while (par[size_t(a)] != a) {
            par[size_t(a)] = par[size_t(par[size_t(a)])];
            a = par[size_t(a)];
        }
        return a;
    };
    for (int32_t i = 0; i < m; ++i) {
        const int32_t a = find(u[i]), b = find(v[i]);
        if (a == b) {
            err = "edge " + std::to_string(i) + " closes a cycle (or repeats an edge)";
            return TFI_ERR_NOT_TREE;
        }
        par[size_t(a)] = b;
    }
    // CSR, neighbours ascending
    // (degrees and slots by atomic counters; each list is sorted below, so the
    // order in which the slots are claimed does not matter)
    hp.ptr.assign(size_t(n) + 1, 0);
    constexpr int32_t kEdgeBlock = 1 << 16;
    const size_t neb = size_t((int64_t(m) + kEdgeBlock - 1) / kEdgeBlock);
    {
        std::vector<std::atomic<int64_t>> cnt(static_cast<size_t>(n));
        for (auto &c : cnt) c.store(0, std::memory_order_relaxed);
        parallel_for(neb, [&](size_t b) {
            const int32_t i1 = std::min(m, int32_t(b) * kEdgeBlock + kEdgeBlock);
            for (int32_t i = int32_t(b) * kEdgeBlock; i < i1; ++i) {
                cnt[size_t(u[i])].fetch_add(1, std::memory_order_relaxed);
                cnt[size_t(v[i])].fetch_add(1, std::memory_order_relaxed);
            }
        });
        for (int32_t i = 0; i < n; ++i) hp.ptr[size_t(i) + 1] = hp.ptr[size_t(i)] + cnt[size_t(i)].load(std::memory_order_relaxed);
    }
    {
        std::vector<std::pair<int32_t, int64_t>> tmp(size_t(2 * int64_t(m)));
        std::vector<std::atomic<int64_t>> fill(static_cast<size_t>(n));
        for (int32_t i = 0; i < n; ++i) fill[size_t(i)].store(hp.ptr[size_t(i)], std::memory_order_relaxed);
        parallel_for(neb, [&](size_t b) {
            const int32_t i1 = std::min(m, int32_t(b) * kEdgeBlock + kEdgeBlock);
            for (int32_t i = int32_t(b) * kEdgeBlock; i < i1; ++i) {
                tmp[size_t(fill[size_t(u[i])].fetch_add(1, std::memory_order_relaxed))] =
                    std::make_pair(int32_t(v[i]), q[size_t(i)]);
                tmp[size_t(fill[size_t(v[i])].fetch_add(1, std::memory_order_relaxed))] =
                    std::make_pair(int32_t(u[i]), q[size_t(i)]);
            }
        });
        hp.adj.resize(tmp.size());
        hp.qlen.resize(tmp.size());
        // each vertex's list sorted by neighbour (distinct in a forest), in blocks of vertices
        constexpr int32_t kBlock = 1 << 14;
        parallel_for(size_t((n + kBlock - 1) / kBlock), [&](size_t blk) {
            const int32_t a0 = int32_t(blk) * kBlock, a1 = std::min(n, a0 + kBlock);
            for (int32_t a = a0; a < a1; ++a) {
                std::sort(tmp.begin() + hp.ptr[size_t(a)], tmp.begin() + hp.ptr[size_t(a) + 1]);
                for (int64_t e = hp.ptr[size_t(a)]; e < hp.ptr[size_t(a) + 1]; ++e) {
                    hp.adj[size_t(e)] = tmp[size_t(e)].first;
                    hp.qlen[size_t(e)] = tmp[size_t(e)].second;
                }
            }
        });
    }
    // trees of the forest, each as an ascending vertex list (tree order = smallest
    // vertex): number each union-find set at its smallest vertex, then place the
    // vertices by tree in ascending order (a counting sort)
    std::vector<int32_t> tree_of(static_cast<size_t>(n));
    std::vector<int32_t> root_tree(size_t(n), -1);
    std::vector<int64_t> tsize;
    for (int32_t x = 0; x < n; ++x) {
        const int32_t r = find(x);
        if (root_tree[size_t(r)] < 0) {
            root_tree[size_t(r)] = int32_t(tsize.size());
            tsize.push_back(0);
        }
        tree_of[size_t(x)] = root_tree[size_t(r)];
        ++tsize[size_t(tree_of[size_t(x)])];
    }
    std::vector<std::vector<int32_t>> trees(tsize.size());
    for (size_t t = 0; t < trees.size(); ++t) trees[t].reserve(size_t(tsize[t]));
    for (int32_t x = 0; x < n; ++x) trees[size_t(tree_of[size_t(x)])].push_back(x);
    std::vector<int32_t>().swap(par);
    std::vector<int32_t>().swap(root_tree);
    if (trees.size() <= 1) {
        Builder b(hp, true);
        if (int rc = b.run(err)) return rc;
    } else if (int rc = plan_forest(hp, trees, err)) {
        return rc;
    }
    std::vector<int32_t> roots(trees.size());
    for (size_t t = 0; t < trees.size(); ++t) roots[t] = trees[t][0];
    if (int rc = flatten(hp, roots, err)) return rc;
    hp.plan_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return TFI_OK;
}

}  // namespace tfi
