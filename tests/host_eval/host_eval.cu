// Host build of the CUDA path's per-anchor gradient evaluator (eval_anchor, with its
// compile-time cell tables) and pair decoder, for the CPU test that compares them with the
// oracle: test infrastructure, not part of the library.
#define MSC_HOST_EMULATION 1
#include <cfenv>
#include <cstdint>
#include <vector>

#include "../../paper_2409_17346_gb300/csrc/msc_core.cuh"

// the directed roundings that the device takes from __fsub_ru / __fadd_rd, here from the
// host's IEEE rounding modes (built with -frounding-math)
#ifndef __CUDA_ARCH__
float msc::emu_sub_ru(float a, float b)
{
    const int old = std::fegetround();
    std::fesetround(FE_UPWARD);
    volatile float x = a, y = b;
    volatile float r = x - y;
    std::fesetround(old);
    return r;
}

float msc::emu_add_rd(float a, float b)
{
    const int old = std::fegetround();
    std::fesetround(FE_DOWNWARD);
    volatile float x = a, y = b;
    volatile float r = x + y;
    std::fesetround(old);
    return r;
}
#endif

template <int D>
static void pairs_of(const float *field, const msc::Grid &G, int64_t *rows, uint64_t cap, uint64_t *n_out)
{
    std::vector<uint64_t> code(G.n);
    for (uint32_t p = 0; p < G.n; p++) code[p] = msc::anchor_code<D>(field, G, p);
    unsigned long long count = 0;
    for (uint32_t p = 0; p < G.n; p++) msc::decode_pairs<D>(code.data(), G, p, rows, &count, cap);
    *n_out = count;
}

// the gradient pairs (L, U) of a field as rows of 8 vertex ids (unsorted), as the library
// reports them; rows may be null to count
extern "C" int host_gradient_pairs(const float *field, int nx, int ny, int nz, int64_t *rows, uint64_t cap,
                                   uint64_t *n_out)
{
    const msc::Grid G = msc::make_grid(nx, ny, nz);
    if (nz > 1) pairs_of<3>(field, G, rows, cap, n_out);
    else pairs_of<2>(field, G, rows, cap, n_out);
    return 0;
}

// one C-pass (Sec. 4.3) of the CUDA path's case logic (case_mask, case_apply, add_case) on
// (f, g, state), run anchor by anchor on the host: the target set T and restore set X as
// vertex flags, and the numbers of cases and of cases whose target can still move
template <int D>
static void cpass_of(const float *f, const float *g, const uint8_t *state, const msc::Grid &G, int tier,
                     int exact_fallback, uint8_t *T_out, uint8_t *X_out, uint64_t *ncase, uint64_t *nlive)
{
    using namespace msc;
    const uint32_t n = G.n;
    std::vector<uint64_t> cf(n), cg(n);
    for (uint32_t p = 0; p < n; p++) {
        cf[p] = anchor_code<D>(f, G, p);
        cg[p] = anchor_code<D>(g, G, p);
    }
    std::vector<uint32_t> Tbits((n + 31) / 32), Xbits((n + 31) / 32), Tlist(n), Xlist(n);
    std::vector<uint8_t> st(state, state + n);
    Counters cnt{};
    Ctx c{};
    c.G = G;
    c.tier = tier;
    c.exact_fallback = exact_fallback;
    c.f = f;
    c.g = const_cast<float *>(g);
    c.state = st.data();
    c.code_f = cf.data();
    c.code_g = cg.data();
    c.Tbits = Tbits.data();
    c.Xbits = Xbits.data();
    c.Tlist = Tlist.data();
    c.Xlist = Xlist.data();
    c.cnt = &cnt;
    for (uint32_t p = 0; p < n; p++) {
        uint32_t m = case_mask<D>(c, p, cf[p], cg[p]);
        while (m) {
            const int i = __builtin_ctz(m);
            m &= m - 1;
            case_apply<D>(c, p, i);
        }
    }
    for (uint32_t v = 0; v < n; v++) {
        T_out[v] = (Tbits[v >> 5] >> (v & 31)) & 1u;
        X_out[v] = (Xbits[v >> 5] >> (v & 31)) & 1u;
    }
    *ncase = cnt.ncase;
    *nlive = cnt.nlive;
}

extern "C" int host_cpass(const float *f, const float *g, const uint8_t *state, int nx, int ny, int nz, int tier,
                          int exact_fallback, uint8_t *T_out, uint8_t *X_out, uint64_t *ncase, uint64_t *nlive)
{
    const msc::Grid G = msc::make_grid(nx, ny, nz);
    if (nz > 1) cpass_of<3>(f, g, state, G, tier, exact_fallback, T_out, X_out, ncase, nlive);
    else cpass_of<2>(f, g, state, G, tier, exact_fallback, T_out, X_out, ncase, nlive);
    return 0;
}

// One C-round from (g, state) on the host, in either of the CUDA path's forms; g and state
// are updated in place, and the numbers of targets and restores are returned.
//  fused = 0 (round graphs): the C-pass lists the targets and restores, then every item is
//    edited (edit_prepare / edit_apply);
//  fused = 1 (persistent round kernel): the C-pass reads the pre-round values from gprev and
//    edits each target when it lists it (fuse_target, value only); then the restores; then
//    the new state of every edited target (state_after).
template <int D>
static void round_of(const float *f, const float *fhat, float *g, uint8_t *state, const msc::Grid &G, int tier,
                     int exact_fallback, float xi, int q_max, int fused, uint64_t *nT, uint64_t *nX)
{
    using namespace msc;
    const uint32_t n = G.n;
    std::vector<uint64_t> cf(n), cg(n);
    for (uint32_t p = 0; p < n; p++) {
        cf[p] = anchor_code<D>(f, G, p);
        cg[p] = anchor_code<D>(g, G, p);
    }
    std::vector<uint32_t> Tbits((n + 31) / 32), Xbits((n + 31) / 32), Tlist(n), Xlist(n), Elist(2 * (size_t)n);
    std::vector<float> gprev(g, g + n);
    Counters cnt{};
    Ctx c{};
    c.G = G;
    c.tier = tier;
    c.exact_fallback = exact_fallback;
    c.f = f;
    c.fhat = fhat;
    c.g = g;
    c.gprev = gprev.data();
    c.state = state;
    c.xi = xi;
    c.qmax = q_max;
    c.qcap = q_max;
    c.step = xi / (float)(1 << q_max);
    c.code_f = cf.data();
    c.code_g = cg.data();
    c.Tbits = Tbits.data();
    c.Xbits = Xbits.data();
    c.Tlist = Tlist.data();
    c.Xlist = Xlist.data();
    c.Elist = Elist.data();
    c.cnt = &cnt;
    Ctx cp = c;
    if (fused) {
        cp.g = gprev.data();        // the cases read the pre-round values
        cp.fuse_g = g;              // targets are edited into g as they are listed
    }
    for (uint32_t p = 0; p < n; p++) {
        uint32_t m = case_mask<D>(cp, p, cf[p], cg[p]);
        while (m) {
            const int i = __builtin_ctz(m);
            m &= m - 1;
            case_apply<D>(cp, p, i);
        }
    }
    const uint32_t t = (uint32_t)cnt.nT, x = (uint32_t)cnt.nX;
    if (!fused) {
        for (uint32_t i = 0; i < x + t; i++) {
            uint32_t v;
            if (edit_prepare(c, i, x, v)) edit_apply(c, i, x, v);
        }
    } else {
        for (uint32_t i = 0; i < x; i++) {
            const uint32_t v = Xlist[i];
            if (state[v] != ST_EXACT) {
                g[v] = f[v];
                state[v] = ST_EXACT;
                Elist[cnt.nE++] = v;
            }
        }
        for (uint64_t i = 0; i < cnt.nE; i++) state_after(c, Elist[i]);
    }
    *nT = t;
    *nX = x;
}

extern "C" int host_round(const float *f, const float *fhat, float *g, uint8_t *state, int nx, int ny, int nz, int tier,
                          int exact_fallback, float xi, int q_max, int fused, uint64_t *nT, uint64_t *nX)
{
    const msc::Grid G = msc::make_grid(nx, ny, nz);
    if (nz > 1) round_of<3>(f, fhat, g, state, G, tier, exact_fallback, xi, q_max, fused, nT, nX);
    else round_of<2>(f, fhat, g, state, G, tier, exact_fallback, xi, q_max, fused, nT, nX);
    return 0;
}

// every anchor's packed gradient code
extern "C" int host_codes(const float *field, int nx, int ny, int nz, uint64_t *out)
{
    const msc::Grid G = msc::make_grid(nx, ny, nz);
    for (uint32_t p = 0; p < G.n; p++) out[p] = nz > 1 ? msc::anchor_code<3>(field, G, p) : msc::anchor_code<2>(field, G, p);
    return 0;
}

// the round's refresh set as the edit and mark kernels build it: every vertex v with
// moved[v] != 0 went from g_old[v] to g_new[v] in the round (gprev = g_old there); the
// anchors in the window of each moved vertex whose order against a vertex within two
// edges changed (order_changed) are flagged in dirty_out
// pairwise = 1: as the CUDA path marks them, only the anchors whose windows hold both ends of
// a pair whose order flipped (the window masks of msc::rt_ring_win, OR-ed over the flipped pairs)
template <int D>
static void dirty_of(const float *g_old, const float *g_new, const uint8_t *moved, const msc::Grid &G, int pairwise,
                     uint8_t *dirty_out)
{
    using namespace msc;
    const Tab<D> &T = rt_tab<D>();
    const uint32_t n = G.n;
    std::vector<uint32_t> Tbits((n + 31) / 32), Xbits((n + 31) / 32);
    std::vector<float> gprev(g_old, g_old + n), g(g_new, g_new + n);
    for (uint32_t v = 0; v < n; v++)
        if (moved[v]) Tbits[v >> 5] |= 1u << (v & 31);
    Ctx c{};
    c.G = G;
    c.g = g.data();
    c.gprev = gprev.data();
    c.Tbits = Tbits.data();
    c.Xbits = Xbits.data();
    const RingWin<D> &RW = rt_ring_win<D>();
    for (uint32_t v = 0; v < n; v++) {
        if (!moved[v] || !order_changed<D>(c, v, 0, 1, T.ring)) continue;
        int x, y, z;
        coords(G, v, x, y, z);
        uint64_t mask = ~0ull;
        if (pairwise) {
            // each ring vertex u on its own: a flip of (v, u) adds the anchors that hold both
            mask = 0;
            const float ov = gprev[v], nv = g[v];
            for (int j = 0; j < T.nring; j++) {
                const int ux = x + T.ring[j][0], uy = y + T.ring[j][1], uz = z + T.ring[j][2];
                if (!inside(G, ux, uy, uz)) continue;
                const uint32_t u = vid(G, ux, uy, uz);
                const bool mu = (Tbits[u >> 5] >> (u & 31)) & 1u;
                const float nu = g[u], ou = mu ? gprev[u] : nu;
                if (sos_lt(ov, v, ou, u) != sos_lt(nv, v, nu, u)) mask |= RW.m[j];
            }
        }
        for (int j = 0; j < T.nwin; j++) {
            if (!((mask >> j) & 1ull)) continue;
            const int px = x - T.win[j][0], py = y - T.win[j][1], pz = z - T.win[j][2];
            if (inside(G, px, py, pz)) dirty_out[vid(G, px, py, pz)] = 1;
        }
    }
}

extern "C" int host_dirty(const float *g_old, const float *g_new, const uint8_t *moved, int nx, int ny, int nz,
                          int pairwise, uint8_t *dirty_out)
{
    const msc::Grid G = msc::make_grid(nx, ny, nz);
    if (nz > 1) dirty_of<3>(g_old, g_new, moved, G, pairwise, dirty_out);
    else dirty_of<2>(g_old, g_new, moved, G, pairwise, dirty_out);
    return 0;
}

// The S-pass of the separatrix state (tier 4), run on the host with the CUDA path's device
// functions: the first build (node_bits, path_seed_walks, tri_propagate) on g1, then, when
// g2 differs, the incremental update of every anchor whose code changed (node_bits), then
// the troublemakers (node_targets).  Outputs the target and restore sets and the case count.
template <int D>
static int spass_of(const float *f, const float *g1, const float *g2, const uint8_t *state, const msc::Grid &G,
                    int exact_fallback, uint8_t *T_out, uint8_t *X_out, uint64_t *ncase)
{
    using namespace msc;
    const Tab<D> &T = rt_tab<D>();
    const uint32_t n = G.n;
    constexpr int NTOP = Tab<D>::NTOP;
    std::vector<uint64_t> cf(n), c1(n), c2(n), low(n, 0);
    for (uint32_t p = 0; p < n; p++) {
        cf[p] = anchor_code<D>(f, G, p);
        c1[p] = anchor_code<D>(g1, G, p);
        c2[p] = anchor_code<D>(g2, G, p);
        if (D == 3) {
            // f-lowest vertex slot of each existing triangle (bits 2t) and tetrahedron (24 + 2k)
            int x, y, z;
            coords(G, p, x, y, z);
            const unsigned cin = corner_mask<D>(G, x, y, z);
            for (int t = 0; t < T.NT; t++)
                if ((cin >> T.tB[t]) & 1u) low[p] |= (uint64_t)lowest_of(cell_verts<D>(G, x, y, z, 2, t), f) << (2 * t);
            if ((cin >> 7) & 1u)
                for (int k = 0; k < T.NK; k++)
                    low[p] |= (uint64_t)lowest_of(cell_verts<D>(G, x, y, z, 3, k), f) << (24 + 2 * k);
        }
    }
    std::vector<uint32_t> seeds[3];
    for (uint32_t p = 0; p < n; p++)
        for (int kind = 0; kind < (D == 3 ? 3 : 2); kind++)
            seeds_anchor<D>(cf.data(), G, p, kind, [&](uint32_t u) { seeds[kind].push_back(u); });
    std::vector<uint32_t> ns_v(node_words(n + 4)), ns_top(node_words((size_t)n * NTOP + 4));
    std::vector<uint32_t> ns_tri(node_words((size_t)n * 12 + 4)), ns_dead(node_words((size_t)n * 7 + 4));
    for (auto *a : {&ns_v, &ns_top, &ns_tri, &ns_dead}) std::fill(a->begin(), a->end(), 0x40404040u);
    std::vector<uint32_t> ovf(2 * ((size_t)n * 12 + 4));
    std::vector<uint32_t> Tbits((n + 31) / 32), Xbits((n + 31) / 32), Tlist(n), Xlist(n);
    std::vector<uint8_t> st(state, state + n);
    Counters cnt{};
    Ctx c{};
    c.G = G;
    c.tier = 4;
    c.exact_fallback = exact_fallback;
    c.f = f;
    c.g = const_cast<float *>(g2);
    c.state = st.data();
    c.code_f = cf.data();
    c.low_f = low.data();
    c.code_g = c1.data();
    c.Tbits = Tbits.data(); c.Xbits = Xbits.data(); c.Tlist = Tlist.data(); c.Xlist = Xlist.data();
    c.cnt = &cnt;
    c.ns_v = ns_v.data(); c.ns_top = ns_top.data(); c.ns_tri = ns_tri.data(); c.ns_dead = ns_dead.data();
    c.ovf_out = ovf.data();
    c.ovf_cap = (uint32_t)(ovf.size() / 2);
    auto drain = [&]() {
        while (cnt.novf) {
            std::vector<uint32_t> items(ovf.begin(), ovf.begin() + 2 * cnt.novf);
            cnt.novf = 0;
            for (size_t i = 0; i < items.size(); i += 2) tri_propagate(c, items[i], 0, true, (int)items[i + 1]);
        }
        return cnt.err == 0;
    };
    // first build on g1
    for (uint32_t p = 0; p < n; p++) node_bits<D>(c, p, true);
    for (int kind = 0; kind < 2; kind++)
        path_seed_walks<D, 4>(c, kind, seeds[kind].data(), (uint32_t)seeds[kind].size(), 0, 1);   // one warp of one lane
    if (D == 3)
        for (uint32_t u : seeds[2]) {
            const int32_t o = node_or(c.ns_tri, u, NS_SEED);
            if (o & NS_SEED) continue;
            const int dv = tri_passes(o | NS_SEED) - tri_passes(o);
            if (dv) tri_propagate(c, u, dv, false, 0);
        }
    if (!drain()) return 1;
    // the update to g2: every anchor whose code changed
    c.code_g = c2.data();
    for (uint32_t p = 0; p < n; p++)
        if (c1[p] != c2[p]) node_bits<D>(c, p, false);
    if (!drain()) return 1;
    cnt = Counters{};
    for (uint32_t p = 0; p < n; p++) node_targets<D>(c, p);
    for (uint32_t v = 0; v < n; v++) {
        T_out[v] = (Tbits[v >> 5] >> (v & 31)) & 1u;
        X_out[v] = (Xbits[v >> 5] >> (v & 31)) & 1u;
    }
    *ncase = cnt.ncase;
    return 0;
}

extern "C" int host_spass(const float *f, const float *g1, const float *g2, const uint8_t *state, int nx, int ny,
                          int nz, int exact_fallback, uint8_t *T_out, uint8_t *X_out, uint64_t *ncase)
{
    const msc::Grid G = msc::make_grid(nx, ny, nz);
    return nz > 1 ? spass_of<3>(f, g1, g2, state, G, exact_fallback, T_out, X_out, ncase)
                  : spass_of<2>(f, g1, g2, state, G, exact_fallback, T_out, X_out, ncase);
}

// Eq. 2 as the edit kernel applies it: out_g[v * K + k] and out_state[...] after k = 0 (the
// re-clamped base) .. K - 1 edits of vertex v, K = q_max + 2 (quantised) or 0xEF + 2
// (floating edits, edit_mode 1: no cap on the steps but the state byte's)
extern "C" int host_edit_sequence(const float *f, const float *fhat, uint32_t n, float xi, int q_max, int edit_mode,
                                  float *out_g, uint8_t *out_state)
{
    using namespace msc;
    std::vector<float> g(n);
    std::vector<uint8_t> st(n, 0);
    Ctx c{};
    c.f = f;
    c.fhat = fhat;
    c.g = g.data();
    c.state = st.data();
    c.xi = xi;
    c.qmax = q_max;
    c.qcap = edit_mode ? 0xEF : q_max;
    c.step = xi / (float)(1 << q_max);
    const int K = c.qcap + 2;
    for (uint32_t v = 0; v < n; v++) {
        g[v] = clamp_base(f[v], fhat[v], xi);
        out_g[(size_t)v * K] = g[v];
        out_state[(size_t)v * K] = 0;
        for (int k = 1; k < K; k++) {
            if (st[v] <= c.qcap) edit_apply(c, 1, 0, v);   // a quantised-step item (not a restore)
            out_g[(size_t)v * K + k] = g[v];
            out_state[(size_t)v * K + k] = st[v];
        }
    }
    return 0;
}

// The tier-3 S-pass (terminal mode) with the CUDA path's walks (desc_walk, asc_walk and
// their visited sets) on (f, g, state): the target and restore sets
template <int D>
static void spass_t3_of(const float *f, const float *g, const uint8_t *state, const msc::Grid &G, int exact_fallback,
                        uint8_t *T_out, uint8_t *X_out)
{
    using namespace msc;
    constexpr int NTOP = Tab<D>::NTOP;
    const uint32_t n = G.n;
    std::vector<uint64_t> cf(n), cg(n);
    for (uint32_t p = 0; p < n; p++) {
        cf[p] = anchor_code<D>(f, G, p);
        cg[p] = anchor_code<D>(g, G, p);
    }
    std::vector<uint32_t> seeds[2];
    for (uint32_t p = 0; p < n; p++)
        for (int kind = 0; kind < 2; kind++) seeds_anchor<D>(cf.data(), G, p, kind, [&](uint32_t u) { seeds[kind].push_back(u); });
    std::vector<uint32_t> vis_v((n + 31) / 32), vis_top(((size_t)n * NTOP + 31) / 32);
    std::vector<uint32_t> Tbits((n + 31) / 32), Xbits((n + 31) / 32), Tlist(n), Xlist(n);
    std::vector<uint8_t> st(state, state + n);
    Counters cnt{};
    Ctx c{};
    c.G = G;
    c.tier = 3;
    c.exact_fallback = exact_fallback;
    c.f = f;
    c.g = const_cast<float *>(g);
    c.state = st.data();
    c.code_f = cf.data();
    c.code_g = cg.data();
    c.Tbits = Tbits.data(); c.Xbits = Xbits.data(); c.Tlist = Tlist.data(); c.Xlist = Xlist.data();
    c.vis_v = vis_v.data();
    c.vis_top = vis_top.data();
    c.cnt = &cnt;
    for (uint32_t u : seeds[0]) desc_walk<D>(c, u);
    for (uint32_t b : seeds[1]) asc_walk<D>(c, b);
    for (uint32_t v = 0; v < n; v++) {
        T_out[v] = (Tbits[v >> 5] >> (v & 31)) & 1u;
        X_out[v] = (Xbits[v >> 5] >> (v & 31)) & 1u;
    }
}

extern "C" int host_spass_t3(const float *f, const float *g, const uint8_t *state, int nx, int ny, int nz,
                             int exact_fallback, uint8_t *T_out, uint8_t *X_out)
{
    const msc::Grid G = msc::make_grid(nx, ny, nz);
    if (nz > 1) spass_t3_of<3>(f, g, state, G, exact_fallback, T_out, X_out);
    else spass_t3_of<2>(f, g, state, G, exact_fallback, T_out, X_out);
    return 0;
}
