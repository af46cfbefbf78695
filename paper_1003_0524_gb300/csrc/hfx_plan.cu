// hfx_plan.cu -- the build engine: one cached plan per input structure.
//
// A plan holds everything a build needs that depends only on the structure of
// the inputs (plane-wave and aux lists, band windows, the set of k to build,
// the device buffers the inputs live in): the batches of (k, q) pairs, every
// table every kernel of every batch reads (uploaded once, in one device
// allocation), the layout of the scratch buffers, and, after the first build,
// the whole launch sequence captured as one CUDA graph.  A build then is the
// replay of that graph (or, with keep_products or without graphs, the same
// launch sequence issued directly): no host work, no host synchronisation
// and no table upload per batch.
//
// Batches.  The (k, q) pairs are taken k-major (every q of one k, then the
// next k) and cut into batches whose working buffers (projections Z, Y = v Z
// and their slices, the raw Z^H Y tiles, and the sliced step-function products
// of the batch's k) fit the device; a batch holds whole pairs, so the k points
// of one q may fall into several batches.  Inside a batch the columns are laid
// out q-major (every pair of one q contiguous), which is what the Coulomb
// apply needs (one v_t(q) per column range).  The q sum of Eq. (vec-mat-vec)
// is accumulated per k in FP64 in batch order, ascending q inside a batch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "hfx_internal.cuh"

namespace hfx {

namespace {

long long rup(long long x, long long m) { return (x + m - 1) / m * m; }

template <typename T> T *at(void *base, size_t off) { return reinterpret_cast<T *>(reinterpret_cast<char *>(base) + off); }

struct Geometry {                 // integer boxes of the interstitial convolution
    int tlo[3], tdim[3];          // T_n(K) box: K = G + G1 - G0
    int dlo[3], ddim[3];          // Theta box: K - G2
};

Geometry boxes(hfx_ctx *ctx) {
    Geometry g;
    int amin[3], amax[3], pmin[3], pmax[3];
    for (int x = 0; x < 3; ++x) { amin[x] = pmin[x] = 1 << 29; amax[x] = pmax[x] = -(1 << 29); }
    for (auto &q : ctx->qp)
        for (size_t i = 0; i < q.G.size(); ++i) { int x = i % 3; amin[x] = std::min(amin[x], q.G[i]); amax[x] = std::max(amax[x], q.G[i]); }
    for (auto &k : ctx->kp)
        for (size_t i = 0; i < k.G.size(); ++i) { int x = i % 3; pmin[x] = std::min(pmin[x], k.G[i]); pmax[x] = std::max(pmax[x], k.G[i]); }
    for (int x = 0; x < 3; ++x) {
        if (amin[x] > amax[x]) { amin[x] = amax[x] = 0; }
        g.tlo[x] = amin[x] + pmin[x];          // -G0 in {0, 1}
        g.tdim[x] = (amax[x] + pmax[x] + 1) - g.tlo[x] + 1;
        g.dlo[x] = g.tlo[x] - pmax[x];
        g.ddim[x] = (g.tlo[x] + g.tdim[x] - 1 - pmin[x]) - g.dlo[x] + 1;
    }
    return g;
}

// band block of the Z^H Y tiles: a multiple of 8 up to 64.  A tile's MMA work
// and operand bytes grow with NB (its 128-row A operand is padded), so take the
// NB with the least nblk^2 * NB.
int pick_nb_zhy(int nb_max) {
    int NB = 8;
    long long best = 1LL << 60;
    for (int nbc = 8; nbc <= 64; nbc += 8) {
        long long nblk = (nb_max + nbc - 1) / nbc, cost = nblk * nblk * nbc;
        if (cost < best || (cost == best && nbc > NB)) { best = cost; NB = nbc; }
    }
    return NB;
}

// FNV-1a
struct Hasher {
    uint64_t h = 1469598103934665603ULL;
    void mix(const void *d, size_t n) {
        const unsigned char *c = static_cast<const unsigned char *>(d);
        for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ULL;
    }
    template <typename T> void val(const T &v) { mix(&v, sizeof(v)); }
};

}  // namespace

void record_event(cudaEvent_t e, cudaStream_t st) {
    // inside a stream capture the record becomes an event node of the graph
    // (timed at every replay); outside it is a plain record
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else
        cudaEventRecord(e, st);
}

void fold_kq(const hfx_ctx *ctx, int ik, int iq, int *ikp, int *g0) {
    const int *M = ctx->sys.mesh;
    int jk[3] = {ik / (M[1] * M[2]), (ik / M[2]) % M[1], ik % M[2]};
    int jq[3] = {iq / (M[1] * M[2]), (iq / M[2]) % M[1], iq % M[2]};
    int jp[3];
    for (int x = 0; x < 3; ++x) {
        int d = jk[x] - jq[x];
        jp[x] = ((d % M[x]) + M[x]) % M[x];
        g0[x] = (d - jp[x]) / M[x];
    }
    *ikp = (jp[0] * M[1] + jp[1]) * M[2] + jp[2];
}

struct BatchPlan {
    std::vector<int> qs;              // distinct q of the batch (QDesc order)
    std::vector<QDesc> qd;
    std::vector<PairDesc> pairs;      // q-major
    long long ncols = 0, maxcols = 0, praw_tot = 0;
    int nklist = 0;
    size_t o_pairs = 0, o_qd = 0, o_kpair = 0, o_praw = 0, o_klist = 0, o_kstart = 0, o_klp = 0, o_vb = 0, o_vd = 0;
    size_t o_zg1 = 0, o_zg2 = 0, o_g1t = 0, o_g2t = 0;
    int n_g1t = 0, n_g2t = 0, maxM1 = 0, maxN1 = 0, mx2 = 0;
    ZipwBatch zipw;
    ZmtBatch zmt;
    std::vector<std::pair<int, const double2 *>> overrides;   // (pair, caller's Z)
    cudaEvent_t ev[11] = {};
};

struct BuildPlan {
    uint64_t sig = 0;
    std::vector<int> kset;
    bool tc = false;
    Geometry geo{};
    long long tbox = 0, dbox = 0, RSc = 0;
    int N0 = 0, sparse = 0, nb_max = 0, no_max = 0, npw_max = 0, maxD = 0, N0pad = 0, Dpad = 0, HS = 0, RS = 0, MP = 0;
    int NB = 8;
    size_t o_A = 0, o_c = 0, o_G = 0, o_Ga = 0, o_npw = 0, o_nb = 0, o_no = 0, o_B = 0, o_T = 0, o_vacc = 0, o_V = 0;
    bool kp = false;                  // the k.p term at q = 0 is added
    bool inv = false;                 // inversion symmetry: packed real bands (Sec. III.D)
    size_t o_sym = 0;                 // row operations Z' = S^H Z
    int nsym = 0;
    size_t o_eps = 0, o_p = 0, o_kp = 0;
    size_t vtot = 0;
    TpPlan tp;
    ZmtPlan zmt;
    ZipwBuild zipw;
    size_t zipw_tq_off = 0;           // offset of the T slices inside s_zipw
    std::vector<BatchPlan> batches;
    void *d_tab = nullptr;            // every table of the plan
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool graph_failed = false;
    int runs = 0;                     // builds executed with this plan
    int nlaunch = 0;
    cudaEvent_t e_start = nullptr, e_fin0 = nullptr, e_end = nullptr;
    double flops = 0, fl_apply = 0, fl_apply_exec = 0, fl_zhy = 0, fl_zipw = 0;
    int npairs_total = 0;
    int device = 0;

    ~BuildPlan() {
        cudaSetDevice(device);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        for (auto &b : batches)
            for (auto e : b.ev)
                if (e) cudaEventDestroy(e);
        if (e_start) cudaEventDestroy(e_start);
        if (e_fin0) cudaEventDestroy(e_fin0);
        if (e_end) cudaEventDestroy(e_end);
        if (d_tab) cudaFree(d_tab);
    }
};

namespace {

Scratch *build_scratch(hfx_ctx *ctx, int i) {
    Scratch *all[] = {&ctx->s_theta, &ctx->s_thpsi, &ctx->s_B,   &ctx->s_zc,   &ctx->s_zs,  &ctx->s_ys,  &ctx->s_y64,
                      &ctx->s_praw,  &ctx->s_vacc,  &ctx->s_xexp, &ctx->s_zipw, &ctx->s_cgT, &ctx->s_cgZ};
    return i < (int)(sizeof(all) / sizeof(all[0])) ? all[i] : nullptr;
}

void free_build_scratch(hfx_ctx *ctx) {
    for (int i = 0; Scratch *s = build_scratch(ctx, i); ++i) {
        if (s->p) cudaFree(s->p);
        s->p = nullptr;
        s->bytes = 0;
    }
}

uint64_t plan_signature(hfx_ctx *ctx, const std::vector<int> &kset) {
    Hasher h;
    h.val(ctx->struct_epoch);
    h.mix(kset.data(), kset.size() * sizeof(int));
    h.val(ctx->opt.precision);
    h.val(ctx->opt.work_bytes);
    h.val(ctx->opt.tile_nb_zhy);
    h.val(ctx->opt.tile_nb_zipw);
    h.val(ctx->opt.q0_term);
    h.val(ctx->q0_bracket);
    h.val(ctx->sparse_used);
    h.val(ctx->N0);
    for (auto &k : ctx->kp) { h.val(k.d_G); h.val(k.d_c); h.val(k.d_A); h.val(k.nb); h.val(k.no); h.val(k.npw); }
    for (auto &q : ctx->qp) { h.val(q.d_G); h.val(q.d_VD); h.val(q.d_VB); h.val(q.nipw); }
    h.val(ctx->d_T); h.val(ctx->d_R); h.val(ctx->d_gaunt); h.val(ctx->d_posf); h.val(ctx->d_err); h.val(ctx->d_Ex);
    h.val(ctx->s_ap.p); h.val(ctx->s_aexp.p);
    h.val(ctx->opt.kp_term); h.val(ctx->opt.kp_deg_tol); h.val(ctx->opt.inversion);
    for (auto &k : ctx->kp) { h.val(k.d_cm); h.val(k.d_Am); h.val(k.nom); }
    for (auto &k : ctx->kp) { h.val(k.d_eps); h.val(k.d_p); h.val(k.d_kp); }
    for (auto &z : ctx->zover) { h.val(z.first); h.val(z.second); }
    return h.h;
}

// ---------------------------------------------------------------- plan build
template <typename R>
int plan_build(hfx_ctx *ctx, const std::vector<int> &kset, BuildPlan &pl) {
    using V = typename C2<R>::T;
    const bool tc = ctx->opt.precision == HFX_PREC_SLICED;
    const hfx_system &s = ctx->sys;
    const int nk = ctx->nk, P = ctx->P, nch = ctx->nch, nmt = ctx->nmt;
    int rc;
    pl.kset = kset;
    pl.tc = tc;
    pl.device = ctx->device;
    pl.N0 = ctx->N0;
    pl.sparse = ctx->sparse_used ? 1 : 0;
    const int N0 = pl.N0, sparse = pl.sparse;
    int naux_max = 0;
    for (auto &q : ctx->qp) { naux_max = std::max(naux_max, nmt + q.nipw); pl.maxD = std::max(pl.maxD, nmt + q.nipw - N0); }
    for (auto &k : ctx->kp) {
        pl.nb_max = std::max(pl.nb_max, k.nb);
        pl.no_max = std::max(pl.no_max, k.nom);   // occupied columns per k' (packed pairs with inversion)
        pl.npw_max = std::max(pl.npw_max, k.npw);
    }
    pl.inv = ctx->opt.inversion != 0;
    pl.RSc = naux_max;
    pl.N0pad = (int)rup(N0, 64);
    pl.Dpad = (int)rup(pl.maxD, 128);
    pl.HS = pl.N0pad + pl.Dpad;
    pl.RS = 2 * pl.HS;
    pl.MP = 2 * pl.Dpad;
    const long long RSc = pl.RSc;
    pl.NB = gemm2_check_nb(ctx->opt.tile_nb_zhy) ? ctx->opt.tile_nb_zhy : pick_nb_zhy(pl.nb_max);
    const int NB = pl.NB;

    // hno: occupied bands (the q->0 and k.p terms); hnom: occupied columns of k' in
    // the projections (with inversion symmetry two real bands share a column)
    std::vector<int> hnpw(nk), hnb(nk), hno(nk), hnom(nk);
    for (int i = 0; i < nk; ++i) {
        hnpw[i] = ctx->kp[i].npw; hnb[i] = ctx->kp[i].nb; hno[i] = ctx->kp[i].no; hnom[i] = ctx->kp[i].nom;
    }
    pl.geo = boxes(ctx);
    pl.tbox = (long long)pl.geo.tdim[0] * pl.geo.tdim[1] * pl.geo.tdim[2];
    pl.dbox = (long long)pl.geo.ddim[0] * pl.geo.ddim[1] * pl.geo.ddim[2];
    if (pl.tbox > (1LL << 26) || pl.dbox > (1LL << 27)) return set_err(ctx, HFX_EUNSUPPORTED, "plane-wave boxes too large");

    // ---- fixed per-build buffers: Theta box, B_k, T_k, the q sums, V^x
    free_build_scratch(ctx);
    size_t bsz = (size_t)s.n_atoms * ctx->nLM * P * ctx->nlmp;
    std::vector<size_t> boff(nk), toff(nk), voff(nk);
    size_t btot = 0, ttot = 0, vtot = 0;
    for (int i = 0; i < nk; ++i) {
        boff[i] = btot; btot += bsz * hnb[i];
        toff[i] = ttot; ttot += (size_t)pl.tbox * hnb[i];
        voff[i] = vtot; vtot += (size_t)hnb[i] * hnb[i];
    }
    pl.vtot = vtot;
    if ((rc = scratch_reserve(ctx, ctx->s_B, btot * sizeof(V))) || (rc = scratch_reserve(ctx, ctx->s_thpsi, ttot * sizeof(V))) ||
        (rc = scratch_reserve(ctx, ctx->s_theta, pl.dbox * sizeof(double2))) ||
        (rc = scratch_reserve(ctx, ctx->s_vacc, vtot * sizeof(double2))))
        return rc;
    if (ctx->V_nb.size() != (size_t)nk) ctx->V_nb.assign(nk, 0);
    for (int i = 0; i < nk; ++i) {
        if (!ctx->d_V[i] || ctx->V_nb[i] != hnb[i]) {   // (re)allocate when the band window changed
            if (ctx->d_V[i]) cudaFree(ctx->d_V[i]);
            ctx->d_V[i] = nullptr;
            if ((rc = cuda_check(ctx, cudaMalloc(&ctx->d_V[i], sizeof(double2) * std::max(1, hnb[i] * hnb[i])), "V^x buffer")))
                return rc;
            ctx->V_nb[i] = hnb[i];
        }
    }
    std::vector<const double2 *> hA(nk), hc(nk);
    std::vector<const int *> hG(nk), hGa(nk);
    std::vector<V *> hB(nk), hT(nk);
    std::vector<double2 *> hvacc(nk), hV(nk);
    for (int i = 0; i < nk; ++i) {
        hA[i] = ctx->kp[i].d_Am; hc[i] = ctx->kp[i].d_cm; hG[i] = ctx->kp[i].d_G; hGa[i] = ctx->qp[i].d_G;
        hB[i] = at<V>(ctx->s_B.p, boff[i] * sizeof(V));
        hT[i] = at<V>(ctx->s_thpsi.p, toff[i] * sizeof(V));
        hvacc[i] = at<double2>(ctx->s_vacc.p, voff[i] * sizeof(double2));
        hV[i] = ctx->d_V[i];
    }
    HostArena tab;
    pl.o_A = tab.put(hA); pl.o_c = tab.put(hc); pl.o_G = tab.put(hG); pl.o_Ga = tab.put(hGa);
    pl.o_npw = tab.put(hnpw); pl.o_nb = tab.put(hnb); pl.o_no = tab.put(hno);
    pl.o_B = tab.put(hB); pl.o_T = tab.put(hT); pl.o_vacc = tab.put(hvacc); pl.o_V = tab.put(hV);
    if (ctx->opt.kp_term) {
        std::vector<const double *> he(nk);
        std::vector<const double2 *> hp(nk);
        std::vector<double2 *> hk(nk);
        for (int i = 0; i < nk; ++i) {
            const KPoint &k = ctx->kp[i];
            if (!k.kp_set || k.kp_nb != k.nb)
                return set_err(ctx, HFX_EMISSING, "kp_term: set_momentum missing for k " + std::to_string(i));
            he[i] = k.d_eps; hp[i] = k.d_p; hk[i] = k.d_kp;
        }
        pl.kp = true;
        pl.o_eps = tab.put(he); pl.o_p = tab.put(hp); pl.o_kp = tab.put(hk);
    }
    if (pl.inv) {
        std::vector<SymOp> ops = sym_row_ops(ctx, N0, sparse);
        pl.nsym = (int)ops.size();
        pl.o_sym = tab.put(ops);
    }

    // ---- per-build products on the tensor cores (plans; their scratch is reserved below)
    if (tc) {
        if ((rc = thetapsi_tc_plan(ctx, kset, pl.geo.ddim, pl.geo.tdim, toff, tab, pl.tp))) return rc;
        std::vector<double2 *> hB2(nk);
        for (int i = 0; i < nk; ++i) hB2[i] = reinterpret_cast<double2 *>(hB[i]);
        if ((rc = zmt_tc_plan(ctx, kset, hB2, RSc, N0, sparse, tab, pl.zmt))) return rc;
        if ((rc = zipw_tc_plan_build(ctx, kset, pl.nb_max, pl.geo.tlo, pl.geo.tdim, ctx->opt.tile_nb_zipw, tab, pl.zipw)))
            return rc;
    }
    const size_t fixed_more = (tc ? pl.tp.scratch_bytes + pl.zmt.scratch_bytes + pl.zipw.scratch_bytes : 0);

    // ---- batches: whole pairs, k-major, within the budget
    size_t budget = ctx->opt.work_bytes;
    if (!budget) {
        size_t fr = 0, totm = 0;
        cudaMemGetInfo(&fr, &totm);
        const size_t reserve = fixed_more + ((size_t)1 << 30) + tab.buf.size() + ((size_t)256 << 20);
        budget = fr > reserve ? (size_t)(0.93 * (double)(fr - reserve)) : 0;
    }
    auto pair_bytes = [&](int ik, int ikp) {
        const long long nc = (long long)hnom[ikp] * hnb[ik];
        size_t praw = tc ? (size_t)((hnb[ik] + NB - 1) / NB) * ((hnb[ik] + NB - 1) / NB) * (2 * NB) * (2 * NB) * sizeof(double)
                         : (size_t)hnb[ik] * hnb[ik] * sizeof(double2);
        size_t b = (size_t)nc * RSc * sizeof(V) + praw + (size_t)nc * RSc * sizeof(double2);
        if (tc) b += (size_t)2 * 4 * nc * pl.RS * sizeof(__nv_bfloat16) + 2 * nc * sizeof(int);
        return b;
    };
    std::vector<std::vector<std::pair<int, int>>> groups;   // (ik, iq) per batch, k-major
    {
        std::vector<std::pair<int, int>> cur;
        std::vector<char> kin(nk, 0);
        size_t used = 0;
        for (int ik : kset)
            for (int iq = 0; iq < nk; ++iq) {
                int ikp, g0[3];
                fold_kq(ctx, ik, iq, &ikp, g0);
                size_t b = pair_bytes(ik, ikp);
                const size_t kb = (tc && !kin[ik]) ? pl.zipw.tq_bytes_per_slot : 0;
                if (!cur.empty() && used + b + kb > budget) {
                    groups.push_back(cur);
                    cur.clear();
                    std::fill(kin.begin(), kin.end(), 0);
                    used = 0;
                }
                const size_t kb2 = (tc && !kin[ik]) ? pl.zipw.tq_bytes_per_slot : 0;
                if (b + kb2 > budget && ctx->opt.work_bytes == 0)
                    return set_err(ctx, HFX_ENOMEM, "one (k, q) pair needs more device memory than is free");
                kin[ik] = 1;
                cur.push_back({ik, iq});
                used += b + kb2;
            }
        if (!cur.empty()) groups.push_back(cur);
    }

    // ---- per-batch layout (columns q-major), flops, scratch sizes
    pl.batches.resize(groups.size());
    long long max_ncols = 0, max_praw = 0;
    size_t max_tq = 0;
    for (size_t bi = 0; bi < groups.size(); ++bi) {
        BatchPlan &bt = pl.batches[bi];
        std::vector<std::pair<int, int>> g = groups[bi];
        std::stable_sort(g.begin(), g.end(), [](const std::pair<int, int> &a, const std::pair<int, int> &b) {
            return a.second < b.second;   // q-major, k order kept inside a q
        });
        long long col = 0;
        for (size_t i = 0; i < g.size(); ++i) {
            const int ik = g[i].first, iq = g[i].second;
            if (bt.qs.empty() || bt.qs.back() != iq) {
                if (!bt.qs.empty()) {
                    QDesc &qp = bt.qd.back();
                    qp.npairs = (int)bt.pairs.size() - qp.pair0;
                    qp.ncols = col - qp.colbase;
                }
                QDesc qd;
                qd.iq = iq;
                qd.nipw = ctx->qp[iq].nipw;
                qd.naux = nmt + qd.nipw;
                qd.D = qd.naux - N0;
                qd.colbase = col;
                qd.pair0 = (int)bt.pairs.size();
                qd.ncols = 0;
                qd.npairs = 0;
                bt.qs.push_back(iq);
                bt.qd.push_back(qd);
            }
            const QDesc &qd = bt.qd.back();
            PairDesc pr;
            pr.ik = ik;
            pr.iq = iq;
            fold_kq(ctx, ik, iq, &pr.ikp, pr.g0);
            pr.nb = hnb[ik];
            pr.no = hnom[pr.ikp];
            pr.col0 = col;
            pr.qslot = (int)bt.qs.size() - 1;
            pr.pad = 0;
            bt.pairs.push_back(pr);
            col += (long long)pr.no * pr.nb;
            // useful flops of the method (sparse form of Fig. 1 where used): 8 per
            // complex multiply-add, or 2 per real one over the m = n_occ(k') real
            // bands with inversion symmetry (Sec. III.D)
            const double m = pl.inv ? hno[pr.ikp] : pr.no, n = pr.nb, f = pl.inv ? 2.0 : 8.0;
            const double nnz = sparse ? (double)qd.D * qd.D + (double)nch * (P * P - 1) : (double)qd.naux * qd.naux;
            pl.flops += f * m * n * (nnz + (double)qd.naux * n) + f * m * n * ctx->nlmp * nmt +
                        f * m * n * qd.nipw * hnpw[pr.ikp];
            pl.fl_apply += f * m * n * (double)qd.D * qd.D;
            // as executed: the upper triangle (sliced path), over the packed columns
            // (two real parts of Y' per column with a real v_t)
            const double mc = pr.no, fe = pl.inv ? 4.0 : 8.0;
            pl.fl_apply_exec += tc ? fe * mc * n * 0.5 * (double)qd.D * (qd.D + 1) : 8.0 * mc * n * (double)qd.D * qd.D;
            pl.fl_zhy += f * m * n * (double)qd.naux * n;
            pl.fl_zipw += f * m * n * (double)qd.nipw * hnpw[pr.ikp];
        }
        if (!bt.qd.empty()) {
            QDesc &qp = bt.qd.back();
            qp.npairs = (int)bt.pairs.size() - qp.pair0;
            qp.ncols = col - qp.colbase;
        }
        bt.ncols = col;
        for (auto &q : bt.qd) bt.maxcols = std::max(bt.maxcols, q.ncols);
        pl.npairs_total += (int)bt.pairs.size();
        max_ncols = std::max(max_ncols, bt.ncols);
        long long praw = 0;
        for (auto &pr : bt.pairs) {
            if (tc) { long long nblk = (pr.nb + NB - 1) / NB; praw += nblk * nblk * (2 * NB) * (2 * NB); }
            else praw += 2LL * pr.nb * pr.nb;
        }
        bt.praw_tot = praw;
        max_praw = std::max(max_praw, praw);
        if (tc) {
            if ((rc = zipw_tc_plan_batch(ctx, pl.zipw, bt.qs, bt.pairs, tab, bt.zipw))) return rc;
            max_tq = std::max(max_tq, bt.zipw.tq_bytes);
        }
    }

    // ---- scratch of the batches and of the tensor-core stages
    const size_t ncol_max = (size_t)std::max<long long>(1, max_ncols);
    if ((rc = scratch_reserve(ctx, ctx->s_zc, ncol_max * RSc * sizeof(V))) ||
        (rc = scratch_reserve(ctx, ctx->s_praw, (size_t)std::max<long long>(1, max_praw) * sizeof(double))) ||
        (rc = scratch_reserve(ctx, ctx->s_y64, ncol_max * RSc * sizeof(double2))))
        return rc;
    if (tc) {
        Layout zl;
        zl.place(pl.zipw.scratch_bytes);
        pl.zipw_tq_off = zl.place(std::max<size_t>(max_tq, 256));
        if ((rc = scratch_reserve(ctx, ctx->s_zs, (size_t)4 * ncol_max * pl.RS * sizeof(__nv_bfloat16))) ||
            (rc = scratch_reserve(ctx, ctx->s_ys, (size_t)4 * ncol_max * pl.RS * sizeof(__nv_bfloat16))) ||
            (rc = scratch_reserve(ctx, ctx->s_xexp, (size_t)2 * ncol_max * sizeof(int))) ||
            (rc = scratch_reserve(ctx, ctx->s_cgT, std::max<size_t>(pl.tp.scratch_bytes, 256))) ||
            (rc = scratch_reserve(ctx, ctx->s_cgZ, std::max<size_t>(pl.zmt.scratch_bytes, 256))) ||
            (rc = scratch_reserve(ctx, ctx->s_zipw, zl.off)))
            return rc;
    }

    // ---- per-batch tables
    const V *Zc = reinterpret_cast<const V *>(ctx->s_zc.p);
    double2 *Y = reinterpret_cast<double2 *>(ctx->s_y64.p);
    double *praw = reinterpret_cast<double *>(ctx->s_praw.p);
    for (BatchPlan &bt : pl.batches) {
        const int npairs = (int)bt.pairs.size(), nq = (int)bt.qs.size();
        std::vector<int> kpair((size_t)nk * nq, -1);
        for (int i = 0; i < npairs; ++i) kpair[(size_t)bt.pairs[i].ik * nq + bt.pairs[i].qslot] = i;
        std::vector<long long> praw_off(npairs);
        long long po = 0;
        for (int i = 0; i < npairs; ++i) {
            praw_off[i] = po;
            if (tc) { long long nblk = (bt.pairs[i].nb + NB - 1) / NB; po += nblk * nblk * (2 * NB) * (2 * NB); }
            else po += 2LL * bt.pairs[i].nb * bt.pairs[i].nb;
        }
        // per-k pair lists (ascending q) for the reduction
        std::vector<int> klist, kstart, klpairs;
        std::vector<char> seen(nk, 0);
        for (auto &pr : bt.pairs) seen[pr.ik] = 1;
        for (int ik : kset) {
            if (!seen[ik]) continue;
            klist.push_back(ik);
            kstart.push_back((int)klpairs.size());
            for (int qsl = 0; qsl < nq; ++qsl) {
                int pi = kpair[(size_t)ik * nq + qsl];
                // a pair without occupied bands at k - q contributes nothing
                if (pi >= 0 && bt.pairs[pi].no > 0) klpairs.push_back(pi);
            }
        }
        kstart.push_back((int)klpairs.size());
        bt.nklist = (int)klist.size();
        std::vector<const double2 *> hVB(nq), hVD(nq);
        for (int i = 0; i < nq; ++i) { hVB[i] = ctx->qp[bt.qs[i]].d_VB; hVD[i] = ctx->qp[bt.qs[i]].d_VD; }
        bt.o_pairs = tab.put(bt.pairs);
        bt.o_qd = tab.put(bt.qd);
        bt.o_kpair = tab.put(kpair);
        bt.o_praw = tab.put(praw_off);
        bt.o_klist = tab.put(klist);
        bt.o_kstart = tab.put(kstart);
        bt.o_klp = tab.put(klpairs);
        bt.o_vb = tab.put(hVB);
        bt.o_vd = tab.put(hVD);
        for (int i = 0; i < npairs; ++i) {
            auto it = ctx->zover.find(std::make_pair(bt.pairs[i].ik, bt.pairs[i].iq));
            if (it != ctx->zover.end()) bt.overrides.push_back({i, it->second});
        }
        if (tc) {
            if ((rc = zmt_tc_plan_batch(ctx, pl.zmt, bt.pairs, RSc, tab, bt.zmt))) return rc;
            std::vector<unsigned char> t1, t2;
            bt.n_g1t = gemm1_tiles(bt.qd.data(), nq, pl.N0pad, pl.inv, t1);
            bt.n_g2t = gemm2_tiles(bt.pairs.data(), npairs, NB, pl.inv && gemm2_real_form(NB), t2);
            bt.o_g1t = tab.put(t1);
            bt.o_g2t = tab.put(t2);
        } else {
            std::vector<ZGemmBatch> g1(nq), g2(npairs);
            for (int i = 0; i < nq; ++i) {
                const QDesc &q = bt.qd[i];
                ZGemmBatch &b = g1[i];
                b.A = ctx->qp[q.iq].d_VD;
                b.B = reinterpret_cast<const double2 *>(Zc) + q.colbase * RSc;
                b.C = Y + q.colbase * RSc + N0;
                b.M = q.D;
                b.N = (int)q.ncols;
                b.K1 = 1;
                b.K2 = q.naux;
                b.sAi = q.naux; b.sAk2 = 1; b.sAk1 = 0;
                b.sBk2 = 1; b.sBk1 = 0; b.sBj = RSc;
                b.sCi = 1; b.sCj = RSc;
                b.conjA = 0;
                bt.maxM1 = std::max(bt.maxM1, b.M);
                bt.maxN1 = std::max(bt.maxN1, b.N);
            }
            for (int i = 0; i < npairs; ++i) {
                const PairDesc &pr = bt.pairs[i];
                const QDesc &q = bt.qd[pr.qslot];
                ZGemmBatch &b = g2[i];
                b.A = reinterpret_cast<const double2 *>(Zc) + pr.col0 * RSc;
                b.B = Y + pr.col0 * RSc;
                b.C = reinterpret_cast<double2 *>(praw + praw_off[i]);
                b.M = pr.nb;
                b.N = pr.nb;
                b.K1 = pr.no;
                b.K2 = q.naux;
                b.sAi = RSc; b.sAk1 = (long long)pr.nb * RSc; b.sAk2 = 1;
                b.sBk1 = (long long)pr.nb * RSc; b.sBk2 = 1; b.sBj = RSc;
                b.sCi = pr.nb; b.sCj = 1;
                b.conjA = 1;
                bt.mx2 = std::max(bt.mx2, pr.nb);
                if (pr.no == 0) { b.K1 = 1; b.K2 = 0; }
            }
            bt.o_zg1 = tab.put(g1);
            bt.o_zg2 = tab.put(g2);
        }
    }

    // ---- upload every table once
    if ((rc = cuda_check(ctx, cudaMalloc(&pl.d_tab, std::max<size_t>(tab.buf.size(), 256)), "plan tables"))) return rc;
    if ((rc = cuda_check(ctx, cudaMemcpy(pl.d_tab, tab.buf.data(), tab.buf.size(), cudaMemcpyHostToDevice), "plan tables")))
        return rc;
    // timing events
    auto mk = [&](cudaEvent_t *e) { return cuda_check(ctx, cudaEventCreate(e), "event"); };
    if ((rc = mk(&pl.e_start)) || (rc = mk(&pl.e_fin0)) || (rc = mk(&pl.e_end))) return rc;
    for (auto &bt : pl.batches)
        for (auto &e : bt.ev)
            if ((rc = mk(&e))) return rc;
    return HFX_OK;
}

// ---------------------------------------------------------------- execution
void rec(hfx_ctx *ctx, cudaEvent_t e) { record_event(e, ctx->stream); }

template <typename R>
int plan_run(hfx_ctx *ctx, BuildPlan &pl, int keep, int fail_wait) {
    using V = typename C2<R>::T;
    const bool tc = pl.tc;
    const hfx_system &s = ctx->sys;
    const int nk = ctx->nk, P = ctx->P, nch = ctx->nch, nmt = ctx->nmt;
    const int N0 = pl.N0, sparse = pl.sparse;
    const long long RSc = pl.RSc;
    char *tab = reinterpret_cast<char *>(pl.d_tab);
    int rc;
    int nl = 0;
    rec(ctx, pl.e_start);
    // step function and the per-k precomputations (every k is some pair's k')
    launch_theta(reinterpret_cast<double2 *>(ctx->s_theta.p), pl.geo.dlo, pl.geo.ddim, ctx->B, ctx->omega, ctx->d_posf,
                 ctx->d_posf + 3 * s.n_atoms, s.n_atoms, ctx->stream);
    ++nl;
    {
        const size_t bsz = (size_t)s.n_atoms * ctx->nLM * P * ctx->nlmp;
        size_t boff = 0, toff = 0;
        std::vector<size_t> bo(nk), to(nk);
        for (int i = 0; i < nk; ++i) { bo[i] = boff; boff += bsz * ctx->kp[i].nb; to[i] = toff; toff += (size_t)pl.tbox * ctx->kp[i].nb; }
        for (int ik : pl.kset) {
            launch_bmat<R>(ctx->kp[ik].d_A, ctx->d_R, ctx->d_T, ctx->d_gaunt, s.n_atoms, s.lmax, s.Lmax, P, ctx->kp[ik].nb,
                           sparse, at<V>(ctx->s_B.p, bo[ik] * sizeof(V)), ctx->stream);
            ++nl;
            if (!tc) {
                launch_thetapsi<R>(reinterpret_cast<double2 *>(ctx->s_theta.p), pl.geo.dlo, pl.geo.ddim, pl.geo.tlo,
                                   pl.geo.tdim, ctx->kp[ik].d_c, ctx->kp[ik].d_G, ctx->kp[ik].nb, ctx->kp[ik].npw,
                                   at<V>(ctx->s_thpsi.p, to[ik] * sizeof(V)), ctx->stream);
                ++nl;
            }
        }
    }
    if ((rc = cuda_check(ctx, cudaGetLastError(), "per-k kernels"))) return rc;
    if (tc) {
        if ((rc = thetapsi_tc_run(ctx, pl.tp, tab, reinterpret_cast<char *>(ctx->s_cgT.p),
                                  reinterpret_cast<double2 *>(ctx->s_theta.p), pl.geo.dlo, pl.geo.ddim, pl.geo.tlo,
                                  pl.geo.tdim, reinterpret_cast<double2 *>(ctx->s_thpsi.p), &nl)) ||
            (rc = zmt_tc_run_prepare(ctx, pl.zmt, tab, reinterpret_cast<char *>(ctx->s_cgZ.p), &nl)) ||
            (rc = zipw_tc_run_build(ctx, pl.zipw, tab, reinterpret_cast<char *>(ctx->s_zipw.p),
                                    reinterpret_cast<const double2 *const *>(tab + pl.o_c),
                                    reinterpret_cast<const int *const *>(tab + pl.o_G),
                                    reinterpret_cast<const int *>(tab + pl.o_npw),
                                    reinterpret_cast<const double2 *const *>(tab + pl.o_T),
                                    reinterpret_cast<const int *>(tab + pl.o_nb))))
            return rc;
        nl += 2;
    }
    cudaMemsetAsync(ctx->s_vacc.p, 0, pl.vtot * sizeof(double2), ctx->stream);

    V *Zc = reinterpret_cast<V *>(ctx->s_zc.p);
    double *praw = reinterpret_cast<double *>(ctx->s_praw.p);
    for (BatchPlan &bt : pl.batches) {
        const int npairs = (int)bt.pairs.size(), nq = (int)bt.qs.size();
        const PairDesc *d_pairs = reinterpret_cast<const PairDesc *>(tab + bt.o_pairs);
        const QDesc *d_qd = reinterpret_cast<const QDesc *>(tab + bt.o_qd);
        const long long *d_praw_off = reinterpret_cast<const long long *>(tab + bt.o_praw);
        rec(ctx, bt.ev[0]);
        // ---- stage 1: projections
        if (tc) {
            if ((rc = zmt_tc_run_batch(ctx, pl.zmt, bt.zmt, tab, reinterpret_cast<char *>(ctx->s_cgZ.p),
                                       reinterpret_cast<double2 *>(Zc), &nl)))
                return rc;
        } else {
            launch_zmt<R>(d_pairs, npairs, d_qd, reinterpret_cast<V *const *>(tab + pl.o_B),
                          reinterpret_cast<const double2 *const *>(tab + pl.o_A), ctx->d_posf, s.mesh, s.n_atoms, ctx->nLM, P,
                          ctx->nlmp, N0, sparse, pl.no_max, Zc, RSc, ctx->stream);
            ++nl;
        }
        rec(ctx, bt.ev[1]);
        if (tc && sizeof(R) == 8) {
            // the G-major output plane of the interstitial kernel lives in the Y buffer,
            // which is free until the Coulomb apply
            int max_nipw = 0;
            for (auto &q : bt.qd) max_nipw = std::max(max_nipw, q.nipw);
            if ((rc = zipw_tc_run_batch(ctx, pl.zipw, bt.zipw, tab, reinterpret_cast<char *>(ctx->s_zipw.p),
                                        at<__nv_bfloat16>(ctx->s_zipw.p, pl.zipw_tq_off), d_pairs,
                                        reinterpret_cast<const double2 *const *>(tab + pl.o_T),
                                        reinterpret_cast<const int *>(tab + pl.o_nb), reinterpret_cast<double2 *>(Zc), RSc,
                                        reinterpret_cast<double2 *>(ctx->s_y64.p), bt.ncols, d_qd, nq, bt.maxcols, max_nipw,
                                        bt.ev[2], bt.ev[3], &nl)))
                return rc;
        } else {
            rec(ctx, bt.ev[2]);
            rc = launch_zipw<R>(d_pairs, reinterpret_cast<const int *>(tab + bt.o_kpair), nk, pl.nb_max, d_qd, nq,
                                reinterpret_cast<V *const *>(tab + pl.o_T), pl.geo.tlo, pl.geo.tdim,
                                reinterpret_cast<const double2 *const *>(tab + pl.o_c),
                                reinterpret_cast<const int *const *>(tab + pl.o_G), reinterpret_cast<const int *>(tab + pl.o_npw),
                                pl.npw_max, reinterpret_cast<const int *const *>(tab + pl.o_Ga),
                                reinterpret_cast<const int *>(tab + pl.o_nb), ctx->omega, nmt, Zc, RSc, ctx->stream);
            if (rc) return set_err(ctx, rc, "interstitial kernel does not fit this size");
            rec(ctx, bt.ev[3]);
            ++nl;
        }
        if (pl.inv) {   // Z' = S^H Z on the MT rows (Sec. III.D)
            launch_sym_rows<V>(Zc, RSc, bt.ncols, reinterpret_cast<const SymOp *>(tab + pl.o_sym), pl.nsym, ctx->stream);
            ++nl;
        }
        rec(ctx, bt.ev[4]);
        for (auto &ov : bt.overrides) {
            const PairDesc &pr = bt.pairs[ov.first];
            launch_override<R>(ov.second, pr, bt.qd[pr.qslot].naux, ctx->d_T, s.n_atoms, s.Lmax, P, N0, sparse, Zc, RSc, nmt,
                               ctx->stream);
            ++nl;
        }
        if ((rc = cuda_check(ctx, cudaGetLastError(), "projection kernels"))) return rc;
        if (keep) {
            for (int i = 0; i < npairs; ++i) {
                const PairDesc &pr = bt.pairs[i];
                int naux = bt.qd[pr.qslot].naux;
                auto key = std::make_pair(pr.ik, pr.iq);
                auto it = ctx->zkeep.find(key);
                if (it != ctx->zkeep.end()) { cudaFree(it->second); ctx->zkeep.erase(it); }
                double2 *d = nullptr;
                if ((rc = cuda_check(ctx, cudaMalloc(&d, sizeof(double2) * std::max<size_t>(1, (size_t)naux * pr.no * pr.nb)),
                                     "kept projections")))
                    return rc;
                ctx->zkeep[key] = d;
                launch_unpermute<R>(Zc, pr, naux, ctx->d_T, s.n_atoms, s.Lmax, P, N0, sparse, RSc, nmt, d, ctx->stream);
                ++nl;
            }
        }
        rec(ctx, bt.ev[5]);
        // ---- contraction
        if (tc) {
            __nv_bfloat16 *ZS = reinterpret_cast<__nv_bfloat16 *>(ctx->s_zs.p), *YS = reinterpret_cast<__nv_bfloat16 *>(ctx->s_ys.p);
            double2 *Yd = reinterpret_cast<double2 *>(ctx->s_y64.p);
            int *zexp = reinterpret_cast<int *>(ctx->s_xexp.p), *yexp = zexp + bt.ncols;
            launch_slice_cols<V>(Zc, RSc, d_qd, nq, bt.ncols, bt.maxcols, N0, pl.N0pad, pl.Dpad, pl.RS, ZS, zexp, ctx->stream);
            if ((rc = cuda_check(ctx, cudaGetLastError(), "slice kernels"))) return rc;
            rec(ctx, bt.ev[6]);
            // Y' = U Z with U the upper triangle of v_t (half diagonal): the dense
            // rows on the tensor cores, the mu = 0 rows in the channel-block kernel;
            // the q reduction adds P' + P'^H for P' = Z^H Y'
            if ((rc = launch_gemm1_tc(ctx, reinterpret_cast<const __nv_bfloat16 *>(ctx->s_ap.p), (long long)nk * 4 * pl.MP,
                                      reinterpret_cast<const int *>(ctx->s_aexp.p), d_qd, ZS, zexp, Yd, RSc, bt.ncols, N0,
                                      pl.N0pad, pl.Dpad, pl.RS, tab + bt.o_g1t, bt.n_g1t)))
                return rc;
            rec(ctx, bt.ev[7]);
            launch_block_y<V>(d_qd, nq, reinterpret_cast<const double2 *const *>(tab + bt.o_vb), nullptr, Zc, Yd, RSc, P,
                              N0, bt.maxcols, ctx->stream);
            launch_slice_cols<double2>(Yd, RSc, d_qd, nq, bt.ncols, bt.maxcols, N0, pl.N0pad, pl.Dpad, pl.RS, YS, yexp,
                                       ctx->stream);
            rec(ctx, bt.ev[8]);
            if ((rc = launch_gemm2_tc(ctx, ZS, YS, zexp, yexp, bt.ncols, pl.RS, pl.HS, pl.N0pad, d_pairs, d_qd, pl.NB,
                                      d_praw_off, praw, tab + bt.o_g2t, bt.n_g2t, fail_wait,
                                      pl.inv && gemm2_real_form(pl.NB))))
                return rc;
            fail_wait = 0;   // one kernel waits in vain
            rec(ctx, bt.ev[9]);
            nl += 5;
        } else {
            double2 *Yd = reinterpret_cast<double2 *>(ctx->s_y64.p);
            rec(ctx, bt.ev[6]);
            launch_zgemm64(reinterpret_cast<const ZGemmBatch *>(tab + bt.o_zg1), nq, bt.maxM1, bt.maxN1, ctx->stream);
            rec(ctx, bt.ev[7]);
            launch_block64(d_qd, nq, reinterpret_cast<const double2 *const *>(tab + bt.o_vb),
                           reinterpret_cast<const double2 *>(Zc), Yd, RSc, nch, P, N0, bt.maxcols, ctx->stream);
            rec(ctx, bt.ev[8]);
            launch_zgemm64(reinterpret_cast<const ZGemmBatch *>(tab + bt.o_zg2), npairs, bt.mx2, bt.mx2, ctx->stream);
            rec(ctx, bt.ev[9]);
            nl += 3;
            if ((rc = cuda_check(ctx, cudaGetLastError(), "fp64 contraction"))) return rc;
        }
        launch_reduce_pairs(d_pairs, reinterpret_cast<const int *>(tab + bt.o_kstart),
                            reinterpret_cast<const int *>(tab + bt.o_klp), bt.nklist,
                            reinterpret_cast<const int *>(tab + bt.o_klist), praw, d_praw_off, pl.NB,
                            tc ? ((pl.inv && gemm2_real_form(pl.NB)) ? 2 : 1) : 0,
                            pl.inv ? 1 : 0, reinterpret_cast<double2 *const *>(tab + pl.o_vacc),
                            reinterpret_cast<const int *>(tab + pl.o_nb),
                            pl.nb_max, ctx->stream);
        ++nl;
        if ((rc = cuda_check(ctx, cudaGetLastError(), "q reduction"))) return rc;
        rec(ctx, bt.ev[10]);
    }
    rec(ctx, pl.e_fin0);
    if (pl.kp) {
        launch_kp_term(reinterpret_cast<const double *const *>(tab + pl.o_eps), reinterpret_cast<const double2 *const *>(tab + pl.o_p),
                       reinterpret_cast<double2 *const *>(tab + pl.o_kp), reinterpret_cast<const int *>(tab + pl.o_nb),
                       reinterpret_cast<const int *>(tab + pl.o_no), nk, pl.nb_max, nk * ctx->omega, ctx->opt.kp_deg_tol,
                       ctx->stream);
        ++nl;
    }
    launch_finish(reinterpret_cast<double2 *const *>(tab + pl.o_vacc), reinterpret_cast<double2 *const *>(tab + pl.o_V),
                  reinterpret_cast<const int *>(tab + pl.o_nb), reinterpret_cast<const int *>(tab + pl.o_no), nk, pl.nb_max,
                  1.0 / nk, ctx->q0_bracket, ctx->opt.q0_term ? 1 : 0,
                  pl.kp ? reinterpret_cast<double2 *const *>(tab + pl.o_kp) : nullptr, ctx->d_Ex, ctx->stream);
    nl += 2;
    rec(ctx, pl.e_end);
    pl.nlaunch = nl;
    return cuda_check(ctx, cudaGetLastError(), "finish kernels");
}

int check_dev_err(hfx_ctx *ctx) {
    int e = 0;
    int rc = cuda_check(ctx, cudaMemcpy(&e, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost), "error word");
    if (rc) return rc;
    if (e) {
        int z = 0;
        cudaMemcpy(ctx->d_err, &z, sizeof(int), cudaMemcpyHostToDevice);
        return set_err(ctx, e == kDevBadIndex ? HFX_EDEVICE : HFX_ETIMEOUT,
                       "device wait expired or bad index in a kernel (code " + std::to_string(e) + ")");
    }
    return HFX_OK;
}

void fill_stats(hfx_ctx *ctx, BuildPlan &pl, hfx_stats *st, bool graph) {
    if (!st) return;
    std::memset(st, 0, sizeof(*st));
    auto el = [](cudaEvent_t a, cudaEvent_t b) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, a, b) != cudaSuccess) { cudaGetLastError(); return 0.0; }
        return (double)t;
    };
    st->ms_total = el(pl.e_start, pl.e_end);
    for (auto &bt : pl.batches) {
        st->ms_stage1 += el(bt.ev[0], bt.ev[5]);
        st->ms_contract += el(bt.ev[5], bt.ev[10]);
        st->ms_zipw += el(bt.ev[2], bt.ev[3]);
        st->ms_apply += el(bt.ev[6], bt.ev[7]);
        st->ms_zhy += el(bt.ev[8], bt.ev[9]);
    }
    st->ms_finish = el(pl.e_fin0, pl.e_end);
    st->useful_flops = pl.flops;
    st->n_pairs = pl.npairs_total;
    st->n_batches = (int)pl.batches.size();
    st->sparse_used = ctx->sparse_used ? 1 : 0;
    st->n_launches = pl.nlaunch;
    st->flops_apply = pl.fl_apply;
    st->flops_apply_exec = pl.fl_apply_exec;
    st->flops_zhy = pl.fl_zhy;
    st->flops_zipw = pl.fl_zipw;
    st->graph_replayed = graph ? 1 : 0;
    st->tile_nb_zhy = pl.NB;
    st->tile_nb_zipw = pl.zipw.NBt;
}

template <typename R>
int build_with_plan(hfx_ctx *ctx, const std::vector<int> &kset, int keep, hfx_stats *st) {
    int rc;
    const uint64_t sig = plan_signature(ctx, kset);
    if (!ctx->plan || ctx->plan->sig != sig) {
        ctx->plan.reset();
        auto pl = std::make_shared<BuildPlan>();
        if ((rc = plan_build<R>(ctx, kset, *pl))) {
            free_build_scratch(ctx);
            return rc;
        }
        pl->sig = sig;
        ctx->plan = pl;
    }
    BuildPlan &pl = *ctx->plan;
    ctx->lapw_valid = false;
    const int fail = ctx->opt.test_fail_wait;
    ctx->opt.test_fail_wait = 0;
    const bool want_graph = ctx->opt.use_graph && !keep && !fail && !pl.graph_failed;
    bool replayed = false;
    // the first build of a plan runs its launches directly; the second captures
    // them (on a private stream: the caller's may be the legacy default stream)
    // and every later one replays the graph on the caller's stream
    if (want_graph && !pl.exec && pl.runs >= 1) {
        cudaStream_t user = ctx->stream;
        if (!pl.cap_stream && cudaStreamCreateWithFlags(&pl.cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            pl.graph_failed = true;
        }
        if (!pl.graph_failed) {
            ctx->stream = pl.cap_stream;
            cudaError_t e = cudaStreamBeginCapture(pl.cap_stream, cudaStreamCaptureModeThreadLocal);
            int rrc = HFX_OK;
            if (e == cudaSuccess) rrc = plan_run<R>(ctx, pl, 0, 0);
            cudaGraph_t g = nullptr;
            cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(pl.cap_stream, &g) : e;
            ctx->stream = user;
            if (e != cudaSuccess || e2 != cudaSuccess || rrc != HFX_OK || !g ||
                cudaGraphInstantiate(&pl.exec, g, 0) != cudaSuccess) {
                cudaGetLastError();
                if (g) cudaGraphDestroy(g);
                pl.exec = nullptr;
                pl.graph_failed = true;
                ctx->err.clear();
            } else {
                pl.graph = g;
            }
        }
    }
    if (want_graph && pl.exec) {
        if ((rc = cuda_check(ctx, cudaGraphLaunch(pl.exec, ctx->stream), "graph launch"))) return rc;
        replayed = true;
    } else {
        if ((rc = plan_run<R>(ctx, pl, keep, fail))) return rc;
    }
    ++pl.runs;
    if ((rc = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "stream synchronize")) || (rc = check_dev_err(ctx)))
        return rc;
    fill_stats(ctx, pl, st, replayed);
    ctx->built = true;
    return HFX_OK;
}

}  // namespace

int build_run(hfx_ctx *ctx, const std::vector<int> &kset, int keep, hfx_stats *st) {
    return build_with_plan<double>(ctx, kset, keep, st);
}

void plan_release(hfx_ctx *ctx) {
    ctx->plan.reset();
    free_build_scratch(ctx);
}

}  // namespace hfx
