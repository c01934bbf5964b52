// Host-side decomposition planner (see planner.hpp).
#include "planner.hpp"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <deque>
#include <numeric>

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
    uint32_t r = 0;
    for (int i = 0; i < bits; ++i) r |= ((k >> i) & 1u) << (bits - 1 - i);
    return r;
}

// Forward complex DFT in place (radix-2, natural order in and out), FP64.
void fft64(std::complex<double> *a, int lg, int64_t stride) {
    const int64_t n = int64_t(1) << lg;
    for (int64_t i = 0; i < n; ++i) {
        int64_t j = bitrev(uint32_t(i), lg);
        if (i < j) std::swap(a[i * stride], a[j * stride]);
    }
    for (int64_t len = 2; len <= n; len <<= 1) {
        const double ang = -2.0 * M_PI / double(len);
        for (int64_t i = 0; i < n; i += len) {
            for (int64_t k = 0; k < len / 2; ++k) {
                std::complex<double> w(std::cos(ang * double(k)), std::sin(ang * double(k)));
                std::complex<double> x = a[(i + k) * stride];
                std::complex<double> y = a[(i + k + len / 2) * stride] * w;
                a[(i + k) * stride] = x + y;
                a[(i + k + len / 2) * stride] = x - y;
            }
        }
    }
}

class Builder {
public:
    explicit Builder(HostPlan &hp) : hp_(hp), n_(hp.n) {
        member_.assign(size_t(n_), 0);
        onp_.assign(size_t(n_), 0);
        seen_.assign(size_t(n_), 0);
        dist_.assign(size_t(n_), 0);
        par_.assign(size_t(n_), -1);
        sz_.assign(size_t(n_), 0);
        maxchild_.assign(size_t(n_), 0);
    }

    int run(std::string &err) {
        // top-level calls: the trees of the forest, in order of their smallest vertex
        std::deque<std::pair<int32_t, std::vector<int32_t>>> work;
        std::fill(member_.begin(), member_.end(), 1);
        int32_t all_tok = 1;
        std::vector<char> done(size_t(n_), 0);
        for (int32_t s = 0; s < n_; ++s) {
            if (done[size_t(s)]) continue;
            traverse(s, all_tok);
            std::vector<int32_t> comp(order_.begin(), order_.end());
            for (int32_t v : comp) done[size_t(v)] = 1;
            work.emplace_back(0, std::move(comp));
        }
        tok_member_ = 1;
        Decomp dd, dc;
        while (!work.empty()) {
            int32_t level = work.front().first;
            std::vector<int32_t> S = std::move(work.front().second);
            work.pop_front();
            const int32_t mtok = ++tok_member_;
            for (int32_t v : S) member_[size_t(v)] = mtok;
            hp_.n_levels = std::max(hp_.n_levels, level + 1);
            const int32_t minv = *std::min_element(S.begin(), S.end());
            if (int64_t(S.size()) <= hp_.leaf_max) {
                if (int rc = emit_leaf(level, minv, mtok, err)) return rc;
                continue;
            }
            Decomp *D = nullptr;
            int32_t kind = 0;
            if (hp_.policy == TFI_POLICY_CENTROID) {
                decompose(mtok, {centroid(minv, int64_t(S.size()), mtok)}, dc);
                D = &dc;
                kind = 1;
            } else if (hp_.policy == TFI_POLICY_DIAMETER) {
                decompose(mtok, diameter(minv, mtok), dd);
                D = &dd;
            } else {
                decompose(mtok, diameter(minv, mtok), dd);
                decompose(mtok, {centroid(minv, int64_t(S.size()), mtok)}, dc);
                // the centroid wins only with a strictly smaller score (Algorithm 6)
                if (score(int64_t(S.size()), dc) < score(int64_t(S.size()), dd)) {
                    D = &dc;
                    kind = 1;
                } else {
                    D = &dd;
                }
            }
            if (D->H >= kGridMax || D->X.back() >= kGridMax) {
                err = "grid distance beyond 2^30 in a decomposition (choose a larger delta)";
                return TFI_ERR_GRID_OVERFLOW;
            }
            emit_call(level, minv, int32_t(S.size()), kind, *D);
            for (size_t a = 0; a + 1 < D->cptr.size(); ++a) {
                work.emplace_back(level + 1,
                                  std::vector<int32_t>(D->cv.begin() + D->cptr[a], D->cv.begin() + D->cptr[a + 1]));
            }
        }
        return TFI_OK;
    }

private:
    // Traverse the members of S (member == mtok) from s: order_, dist_, par_.
    void traverse(int32_t s, int32_t mtok) {
        const int32_t tok = ++tok_seen_;
        order_.clear();
        order_.push_back(s);
        seen_[size_t(s)] = tok;
        dist_[size_t(s)] = 0;
        par_[size_t(s)] = -1;
        for (size_t h = 0; h < order_.size(); ++h) {
            const int32_t a = order_[h];
            for (int64_t e = hp_.ptr[size_t(a)]; e < hp_.ptr[size_t(a) + 1]; ++e) {
                const int32_t b = hp_.adj[size_t(e)];
                if (member_[size_t(b)] == mtok && seen_[size_t(b)] != tok) {
                    seen_[size_t(b)] = tok;
                    dist_[size_t(b)] = dist_[size_t(a)] + hp_.qlen[size_t(e)];
                    par_[size_t(b)] = a;
                    order_.push_back(b);
                }
            }
        }
    }

    int32_t farthest() const {
        int32_t best = order_[0];
        for (int32_t v : order_) {
            if (dist_[size_t(v)] > dist_[size_t(best)] || (dist_[size_t(v)] == dist_[size_t(best)] && v < best)) best = v;
        }
        return best;
    }

    // Weighted diameter path by two traversals and parent pointers (Algorithm 6, first step).
    std::vector<int32_t> diameter(int32_t minv, int32_t mtok) {
        traverse(minv, mtok);
        const int32_t a = farthest();
        traverse(a, mtok);
        const int32_t b = farthest();
        std::vector<int32_t> path;
        for (int32_t v = b; v != -1; v = par_[size_t(v)]) path.push_back(v);
        std::reverse(path.begin(), path.end());
        return path;
    }

    // Centroid by a rooted traversal and subtree sizes (Algorithm 6, second step).
    int32_t centroid(int32_t minv, int64_t nS, int32_t mtok) {
        traverse(minv, mtok);
        for (int32_t v : order_) {
            sz_[size_t(v)] = 1;
            maxchild_[size_t(v)] = 0;
        }
        for (size_t i = order_.size(); i-- > 1;) {
            const int32_t v = order_[i], p = par_[size_t(v)];
            sz_[size_t(p)] += sz_[size_t(v)];
            maxchild_[size_t(p)] = std::max(maxchild_[size_t(p)], sz_[size_t(v)]);
        }
        int32_t best = -1;
        for (int32_t v : order_) {
            const int64_t big = std::max<int64_t>(nS - sz_[size_t(v)], maxchild_[size_t(v)]);
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
    void decompose(int32_t mtok, std::vector<int32_t> P, Decomp &D) {
        D.clear();
        D.P = std::move(P);
        const int32_t ptok = ++tok_onp_;
        for (int32_t p : D.P) onp_[size_t(p)] = ptok;
        D.X.push_back(0);
        for (size_t j = 1; j < D.P.size(); ++j) D.X.push_back(D.X.back() + edge_len(D.P[j - 1], D.P[j]));
        const int32_t tok = ++tok_seen_;
        for (size_t j = 0; j < D.P.size(); ++j) {
            const int32_t p = D.P[j];
            for (int64_t e = hp_.ptr[size_t(p)]; e < hp_.ptr[size_t(p) + 1]; ++e) {
                const int32_t r = hp_.adj[size_t(e)];
                if (member_[size_t(r)] != mtok || onp_[size_t(r)] == ptok || seen_[size_t(r)] == tok) continue;
                const size_t start = D.cv.size();
                seen_[size_t(r)] = tok;
                D.cv.push_back(r);
                D.cd.push_back(hp_.qlen[size_t(e)]);  // the attaching edge p - r
                int64_t h = 0;
                for (size_t k = start; k < D.cv.size(); ++k) {
                    const int32_t a = D.cv[k];
                    const int64_t da = D.cd[k];
                    h = std::max(h, da);
                    for (int64_t f = hp_.ptr[size_t(a)]; f < hp_.ptr[size_t(a) + 1]; ++f) {
                        const int32_t b = hp_.adj[size_t(f)];
                        if (member_[size_t(b)] == mtok && onp_[size_t(b)] != ptok && seen_[size_t(b)] != tok) {
                            seen_[size_t(b)] = tok;
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
    // with grid distances from that root (subtrees are contiguous ranges).
    int emit_leaf(int32_t level, int32_t minv, int32_t mtok, std::string &err) {
        Leaf lf;
        lf.level = level;
        lf.minv = minv;
        lf.begin = int64_t(hp_.leaf_vtx.size());
        const int32_t tok = ++tok_seen_;
        std::vector<int32_t> &stack = stack_;
        stack.clear();
        stack.push_back(minv);
        seen_[size_t(minv)] = tok;
        dist_[size_t(minv)] = 0;
        par_[size_t(minv)] = -1;
        std::vector<int32_t> kids;
        while (!stack.empty()) {
            const int32_t v = stack.back();
            stack.pop_back();
            if (dist_[size_t(v)] >= kGridMax / 2) {
                err = "grid distance beyond 2^29 inside a leaf (choose a larger delta)";
                return TFI_ERR_GRID_OVERFLOW;
            }
            hp_.leaf_vtx.push_back(v);
            hp_.leaf_dist.push_back(int32_t(dist_[size_t(v)]));
            const int32_t p = par_[size_t(v)];
            hp_.leaf_pdist.push_back(p >= 0 ? int32_t(dist_[size_t(p)]) : 0);
            kids.clear();
            for (int64_t e = hp_.ptr[size_t(v)]; e < hp_.ptr[size_t(v) + 1]; ++e) {
                const int32_t b = hp_.adj[size_t(e)];
                if (member_[size_t(b)] == mtok && seen_[size_t(b)] != tok) {
                    seen_[size_t(b)] = tok;
                    dist_[size_t(b)] = dist_[size_t(v)] + hp_.qlen[size_t(e)];
                    par_[size_t(b)] = v;
                    kids.push_back(b);
                }
            }
            // adjacency is ascending; push in reverse so the smallest child comes next
            for (size_t k = kids.size(); k-- > 0;) stack.push_back(kids[k]);
        }
        lf.end = int64_t(hp_.leaf_vtx.size());
        // leaf diameter by a second traversal from the vertex farthest from the root
        int32_t far = minv;
        int64_t best = -1;
        for (int64_t i = lf.begin; i < lf.end; ++i) {
            if (hp_.leaf_dist[size_t(i)] > best) {
                best = hp_.leaf_dist[size_t(i)];
                far = hp_.leaf_vtx[size_t(i)];
            }
        }
        traverse(far, mtok);
        lf.diam = 0;
        for (int32_t v : order_) lf.diam = std::max(lf.diam, dist_[size_t(v)]);
        hp_.leaves.push_back(lf);
        return TFI_OK;
    }

    HostPlan &hp_;
    int32_t n_;
    std::vector<int32_t> member_, onp_, seen_, par_, order_, stack_;
    std::vector<int64_t> dist_, sz_, maxchild_;
    int32_t tok_member_ = 0, tok_onp_ = 0, tok_seen_ = 0;
};

// Cost model of the two evaluators, per channel, in units of one direct
// multiply-add: direct summation touches every key pair; the FFT path pays a
// forward and an inverse transform of the padded table (both halved by packing
// two channels per complex transform) plus the key scatter and read-back.
constexpr double kFftCostPerPointLog = 3.0;
constexpr double kFftCostPerKey = 4.0;

int flatten(HostPlan &hp, std::string &err) {
    const int64_t R = int64_t(hp.recs.size());
    std::vector<int32_t> rec_akey(size_t(R), -1), rec_bkey(size_t(R), -1);
    hp.key_ptr.assign(1, 0);
    std::vector<int64_t> idx;
    auto add_job = [&](int64_t kb, int64_t ke, int is_comp) {
        Job j{};
        j.kb = kb;
        j.ke = ke;
        j.is_comp = is_comp;
        int32_t maxr = 0, maxx = 0;
        for (int64_t k = kb; k < ke; ++k) {
            maxr = std::max(maxr, hp.key_r[size_t(k)]);
            maxx = std::max(maxx, hp.key_x[size_t(k)]);
        }
        j.maxr = maxr;
        j.maxx = maxx;
        j.lp1 = ceil_log2(2 * int64_t(maxr) + 1);
        j.lp2 = maxx > 0 ? ceil_log2(2 * int64_t(maxx)) : 0;
        const double nk = double(ke - kb);
        const int lg = j.lp1 + j.lp2;
        const double np = std::ldexp(1.0, lg);
        const double cost_fft = kFftCostPerPointLog * np * std::max(1, lg) + kFftCostPerKey * nk;
        j.mode = (lg <= kFftMaxLog && cost_fft < nk * nk) ? 0 : 1;
        hp.jobs.push_back(j);
    };
    for (size_t c = 0; c < hp.calls.size(); ++c) {
        const Call &call = hp.calls[c];
        // A-bins: distinct (depth, coordinate) of the call (Eq. "sumofFFTterms" aggregates A_r[t])
        idx.resize(size_t(call.rec_end - call.rec_begin));
        std::iota(idx.begin(), idx.end(), call.rec_begin);
        std::sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) {
            const Rec &x = hp.recs[size_t(a)], &y = hp.recs[size_t(b)];
            if (x.r != y.r) return x.r < y.r;
            if (x.x != y.x) return x.x < y.x;
            return x.v < y.v;
        });
        const int64_t kb = int64_t(hp.key_r.size());
        for (size_t i = 0; i < idx.size(); ++i) {
            const Rec &rc = hp.recs[size_t(idx[i])];
            if (i == 0 || rc.r != hp.recs[size_t(idx[i - 1])].r || rc.x != hp.recs[size_t(idx[i - 1])].x) {
                if (i) hp.key_ptr.push_back(int32_t(hp.key_vtx.size()));
                hp.key_r.push_back(rc.r);
                hp.key_x.push_back(rc.x);
            }
            hp.key_vtx.push_back(rc.v);
            rec_akey[size_t(idx[i])] = int32_t(hp.key_r.size() - 1);
        }
        hp.key_ptr.push_back(int32_t(hp.key_vtx.size()));
        add_job(kb, int64_t(hp.key_r.size()), 0);
        // b-bins of each component: distinct depths (Eq. "stad-E" profile b_alpha)
        int64_t pos = call.rec_begin + (call.bb_end - call.bb_begin);
        for (int32_t a = call.comp_begin; a < call.comp_end; ++a) {
            const int64_t cb = pos, ce = pos + hp.comps[size_t(a)].size;
            pos = ce;
            idx.resize(size_t(ce - cb));
            std::iota(idx.begin(), idx.end(), cb);
            std::sort(idx.begin(), idx.end(), [&](int64_t p, int64_t q) {
                const Rec &x = hp.recs[size_t(p)], &y = hp.recs[size_t(q)];
                if (x.r != y.r) return x.r < y.r;
                return x.v < y.v;
            });
            const int64_t bk = int64_t(hp.key_r.size());
            for (size_t i = 0; i < idx.size(); ++i) {
                const Rec &rc = hp.recs[size_t(idx[i])];
                if (i == 0 || rc.r != hp.recs[size_t(idx[i - 1])].r) {
                    if (i) hp.key_ptr.push_back(int32_t(hp.key_vtx.size()));
                    hp.key_r.push_back(rc.r);
                    hp.key_x.push_back(0);
                }
                hp.key_vtx.push_back(rc.v);
                rec_bkey[size_t(idx[i])] = int32_t(hp.key_r.size() - 1);
            }
            hp.key_ptr.push_back(int32_t(hp.key_vtx.size()));
            add_job(bk, int64_t(hp.key_r.size()), 1);
        }
    }
    if (hp.key_vtx.size() >= size_t(INT32_MAX)) {
        err = "plan too large for 32-bit bin indices";
        return TFI_ERR_UNSUPPORTED;
    }
    // per vertex: its (A-key, b-key) in every non-leaf call, in level order
    hp.vrec_ptr.assign(size_t(hp.n) + 1, 0);
    for (const Rec &rc : hp.recs) hp.vrec_ptr[size_t(rc.v) + 1]++;
    for (int32_t v = 0; v < hp.n; ++v) hp.vrec_ptr[size_t(v) + 1] += hp.vrec_ptr[size_t(v)];
    hp.vrec_akey.assign(size_t(R), 0);
    hp.vrec_bkey.assign(size_t(R), 0);
    {
        std::vector<int32_t> fill(hp.vrec_ptr.begin(), hp.vrec_ptr.end() - 1);
        for (int64_t i = 0; i < R; ++i) {
            const int32_t v = hp.recs[size_t(i)].v;
            const int32_t slot = fill[size_t(v)]++;
            hp.vrec_akey[size_t(slot)] = rec_akey[size_t(i)];
            hp.vrec_bkey[size_t(slot)] = rec_bkey[size_t(i)];
        }
    }
    // rooted forest for the device distance pass: each tree rooted at its smallest vertex
    {
        hp.k1_parent.assign(size_t(hp.n), -1);
        hp.k1_qpar.assign(size_t(hp.n), 0);
        std::vector<int32_t> hop(size_t(hp.n), 0), queue;
        queue.reserve(size_t(hp.n));
        for (int32_t s0 = 0; s0 < hp.n; ++s0) {
            if (hp.k1_parent[size_t(s0)] >= 0) continue;
            hp.k1_parent[size_t(s0)] = s0;
            queue.clear();
            queue.push_back(s0);
            for (size_t h = 0; h < queue.size(); ++h) {
                const int32_t a = queue[h];
                for (int64_t e = hp.ptr[size_t(a)]; e < hp.ptr[size_t(a) + 1]; ++e) {
                    const int32_t b = hp.adj[size_t(e)];
                    if (hp.k1_parent[size_t(b)] >= 0) continue;
                    hp.k1_parent[size_t(b)] = a;
                    hp.k1_qpar[size_t(b)] = int32_t(hp.qlen[size_t(e)]);
                    hop[size_t(b)] = hop[size_t(a)] + 1;
                    hp.k1_maxhop = std::max(hp.k1_maxhop, hop[size_t(b)]);
                    queue.push_back(b);
                }
            }
        }
        hp.rec_anchor.resize(hp.recs.size());
        hp.rec_p1.resize(hp.recs.size());
        for (const Call &c : hp.calls) {
            const int32_t p1 = hp.bb[size_t(c.bb_begin)];
            for (int64_t i = c.rec_begin; i < c.rec_end; ++i) {
                const Rec &rc = hp.recs[size_t(i)];
                hp.rec_anchor[size_t(i)] =
                    rc.comp >= 0 ? hp.bb[size_t(c.bb_begin + hp.comps[size_t(rc.comp)].anchor_idx)] : rc.v;
                hp.rec_p1[size_t(i)] = p1;
            }
        }
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
        int32_t dmax = 0;
        for (int64_t i = lf.begin; i < lf.end; ++i) {
            hp.leaf_lo[size_t(i)] = int32_t(lf.begin);
            hp.leaf_hi[size_t(i)] = int32_t(lf.end);
            dmax = std::max(dmax, hp.leaf_dist[size_t(i)]);
        }
        (void)dmax;
        need_leaf = std::max<int64_t>(need_leaf, lf.diam);
    }
    if (int64_t(hp.leaf_vtx.size()) > gstart) hp.lgrp_ptr.push_back(int32_t(hp.leaf_vtx.size()));
    // grid samples of f: every direct job and leaf looks values up by index
    int64_t need = need_leaf;
    int64_t need_any = need_leaf;
    for (const Job &j : hp.jobs) {
        const int64_t top = 2 * int64_t(j.maxr) + j.maxx;
        need_any = std::max(need_any, top);
        if (j.mode == 1) need = std::max(need, top);
    }
    if (hp.f.kind == TFI_F_TABLE && need_any >= int64_t(hp.f.table.size())) {
        err = "sampled kernel table shorter than the largest grid distance the plan needs";
        return TFI_ERR_GRID_OVERFLOW;
    }
    hp.ftab_len = need + 1;
    hp.ftab.resize(size_t(hp.ftab_len));
    for (int64_t k = 0; k < hp.ftab_len; ++k) hp.ftab[size_t(k)] = float(hp.f.grid(k, hp.delta));
    // kernel spectra per FFT class: kappa[j][b] = f(j + min(b, P2 - b)); 2D DFT in FP64,
    // scaled by 1/(P1 P2), stored in bit-reversed order along both axes
    hp.spec_class_off.assign(16 * 16, -1);
    std::vector<std::complex<double>> buf;
    for (const Job &j : hp.jobs) {
        if (j.mode != 0) continue;
        const int cls = j.lp1 * 16 + j.lp2;
        if (hp.spec_class_off[size_t(cls)] >= 0) continue;
        const int64_t P1 = int64_t(1) << j.lp1, P2 = int64_t(1) << j.lp2, NP = P1 * P2;
        buf.assign(size_t(NP), 0.0);
        for (int64_t a = 0; a < P1; ++a) {
            for (int64_t b = 0; b < P2; ++b) {
                const int64_t k = a + std::min(b, P2 - b);
                double fv = hp.f.grid(k, hp.delta);
                if (!std::isfinite(fv)) fv = 0.0;  // beyond a sampled table: never read for occupied bins
                buf[size_t(a * P2 + b)] = fv;
            }
        }
        for (int64_t a = 0; a < P1; ++a) fft64(buf.data() + a * P2, j.lp2, 1);
        for (int64_t b = 0; b < P2; ++b) fft64(buf.data() + b, j.lp1, P2);
        hp.spec_class_off[size_t(cls)] = int32_t(hp.spectra.size());
        const size_t off = hp.spectra.size();
        hp.spectra.resize(off + size_t(2 * NP));
        const double scale = 1.0 / double(NP);
        for (int64_t a = 0; a < P1; ++a) {
            for (int64_t b = 0; b < P2; ++b) {
                const std::complex<double> s =
                    buf[size_t(int64_t(bitrev(uint32_t(a), j.lp1)) * P2 + int64_t(bitrev(uint32_t(b), j.lp2)))] * scale;
                hp.spectra[off + size_t(2 * (a * P2 + b))] = float(s.real());
                hp.spectra[off + size_t(2 * (a * P2 + b) + 1)] = float(s.imag());
            }
        }
    }
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

}  // namespace

int build_plan(HostPlan &hp, int32_t n, int32_t m, const int32_t *u, const int32_t *v, const double *w,
               std::string &err) {
    const auto t0 = std::chrono::steady_clock::now();
    hp.n = n;
    // validate and quantise: q_e = max(1, round(w_e / delta)), ties to even
    std::vector<int64_t> q(static_cast<size_t>(m));
    for (int32_t i = 0; i < m; ++i) {
        if (u[i] < 0 || u[i] >= n || v[i] < 0 || v[i] >= n || u[i] == v[i]) {
            err = "edge " + std::to_string(i) + " has an out-of-range endpoint or is a self loop";
            return TFI_ERR_NOT_TREE;
        }
        if (!std::isfinite(w[i]) || !(w[i] > 0.0)) {
            err = "edge " + std::to_string(i) + " has a weight that is not finite and positive";
            return TFI_ERR_WEIGHT;
        }
        const double r = std::nearbyint(w[i] / hp.delta);
        if (!(r < double(kGridMax))) {
            err = "edge length / delta exceeds 2^30";
            return TFI_ERR_GRID_OVERFLOW;
        }
        q[size_t(i)] = std::max<int64_t>(1, int64_t(r));
    }
    // acyclicity by union-find (a forest on n vertices)
    {
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
    }
    // CSR, neighbours ascending
    hp.ptr.assign(size_t(n) + 1, 0);
    for (int32_t i = 0; i < m; ++i) {
        hp.ptr[size_t(u[i]) + 1]++;
        hp.ptr[size_t(v[i]) + 1]++;
    }
    for (int32_t i = 0; i < n; ++i) hp.ptr[size_t(i) + 1] += hp.ptr[size_t(i)];
    {
        std::vector<std::pair<int32_t, int64_t>> tmp(size_t(2 * int64_t(m)));
        std::vector<int64_t> fill(hp.ptr.begin(), hp.ptr.end() - 1);
        for (int32_t i = 0; i < m; ++i) {
            tmp[size_t(fill[size_t(u[i])]++)] = std::make_pair(int32_t(v[i]), q[size_t(i)]);
            tmp[size_t(fill[size_t(v[i])]++)] = std::make_pair(int32_t(u[i]), q[size_t(i)]);
        }
        hp.adj.resize(tmp.size());
        hp.qlen.resize(tmp.size());
        for (int32_t a = 0; a < n; ++a) {
            std::sort(tmp.begin() + hp.ptr[size_t(a)], tmp.begin() + hp.ptr[size_t(a) + 1]);
            for (int64_t e = hp.ptr[size_t(a)]; e < hp.ptr[size_t(a) + 1]; ++e) {
                hp.adj[size_t(e)] = tmp[size_t(e)].first;
                hp.qlen[size_t(e)] = tmp[size_t(e)].second;
            }
        }
    }
    Builder b(hp);
    if (int rc = b.run(err)) return rc;
    if (int rc = flatten(hp, err)) return rc;
    hp.plan_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return TFI_OK;
}

}  // namespace tfi
